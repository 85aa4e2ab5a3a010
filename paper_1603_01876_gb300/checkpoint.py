"""Stage checkpoints of the pipeline, keyed by (scale, seed).

The paper's kernels hand their results to one another through files (the
edge files of Kernels 0 and 1, Sec. IV-A and IV-B); these helpers keep the
same stage boundaries as binary files, so that a long run can stop after a
kernel and resume there:

    save_edges / load_edges    (u, v), before or after Kernel 1
    save_graph / load_graph    Kernel 2's output (every pp_graph array)
    save_ranks / load_ranks    Kernel 3's r after k iterations
    pagerank_resume            Kernel 3 continued from a saved r

Files are numpy .npz archives named s<scale>_seed<seed>_<stage>.npz in the
given directory.  Nothing here is on a timed path; the arrays are copied
through host memory.
"""
import os

import numpy as np
import torch

from . import Graph, graph_lengths, pagerank, rank_update

GRAPH_FIELDS = ("colptr", "rowc", "ovf_key", "ovf_cnt", "d_in", "d_out", "inv_dout32", "inv_dout64", "info", "perm",
                "iperm")


def stage_path(directory, scale, seed, stage):
    return os.path.join(directory, "s%d_seed%d_%s.npz" % (scale, seed, stage))


def _save(path, **arrays):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp.%d.npz" % os.getpid()
    np.savez(tmp, **arrays)
    os.replace(tmp, path)
    return path


def save_edges(directory, scale, seed, u, v, stage="edges"):
    """The edge list (int32 tensors holding uint32 ids); stage "edges" (the
    generator's output) or e.g. "sorted" (Kernel 1's)."""
    return _save(stage_path(directory, scale, seed, stage), scale=np.int64(scale), u=u.cpu().numpy(),
                 v=v.cpu().numpy())


def load_edges(directory, scale, seed, stage="edges", device="cuda"):
    with np.load(stage_path(directory, scale, seed, stage)) as z:
        if int(z["scale"]) != scale:
            raise ValueError("checkpoint holds scale %d" % int(z["scale"]))
        return torch.from_numpy(z["u"]).to(device), torch.from_numpy(z["v"]).to(device)


def save_graph(directory, scale, seed, g, stage="graph"):
    """Every array of Kernel 2's output at its full length (pp_graph_lengths)."""
    if g.scale != scale:
        raise ValueError("graph has scale %d" % g.scale)
    return _save(stage_path(directory, scale, seed, stage), scale=np.int64(g.scale), M=np.int64(g.M),
                 **{f: getattr(g, f).cpu().numpy() for f in GRAPH_FIELDS})


def load_graph(directory, scale, seed, stage="graph", device="cuda"):
    with np.load(stage_path(directory, scale, seed, stage)) as z:
        M, sc = int(z["M"]), int(z["scale"])
        if sc != scale:
            raise ValueError("checkpoint holds scale %d" % sc)
        lens = graph_lengths(M, sc)
        g = Graph(M, sc, device)
        for i, f in enumerate(GRAPH_FIELDS):
            a = z[f]
            if a.shape != (lens[i],):
                raise ValueError("%s has %s elements, expected %d" % (f, a.shape, lens[i]))
            getattr(g, f).copy_(torch.from_numpy(a))
        return g


def save_ranks(directory, scale, seed, r, iterations, stage="ranks"):
    return _save(stage_path(directory, scale, seed, stage), r=r.cpu().numpy(), iterations=np.int64(iterations))


def load_ranks(directory, scale, seed, stage="ranks", device="cuda"):
    """(r, iterations it has had)."""
    with np.load(stage_path(directory, scale, seed, stage)) as z:
        return torch.from_numpy(z["r"]).to(device), int(z["iterations"])


def pagerank_resume(graph, r_k, iters, c=0.85, dtype="fp64", workspace=None, stream=None):
    """Kernel 3 continued for `iters` more iterations from a saved r_k.

    Kernel 3 starts from r0 / norm(r0, 1); every iteration is linear and
    homogeneous in r, so continuing from r_k gives norm(r_k, 1) times the run
    started from r_k.  Both the norm and the rescale run in the library's
    kernels (pp_rank_update); the result equals the uninterrupted run within
    rounding (a few units in the last place)."""
    r_k = r_k.to(torch.float64).contiguous()
    scratch = torch.empty_like(r_k)
    norm = float(rank_update(r_k, 1.0, 0.0, scratch, stream=stream).item())  # r_k >= 0: its sum is its norm
    y = pagerank(graph, r_k, iters, c, dtype, workspace=workspace, stream=stream)
    out = torch.empty_like(y)
    rank_update(y, norm, 0.0, out, stream=stream)
    return out
