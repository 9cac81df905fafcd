"""Worker of the time-slab tests, launched by torch.distributed.run (gloo).

Usage: _slab_worker.py comm OUTDIR
         exercise the host-side communication adapter of the slab (exchange of
         a slice with the ring neighbours, sums over ranks), no GPU needed;
       _slab_worker.py gpu OUTDIR D NX NTAU [device]
         every rank owns its part of the time slices of one lattice (on the
         same GPU when there is one), applies M, M^T and Q to its part of a
         seeded x and solves Q x = b; the parts go to OUTDIR for the test to
         assemble and check against the oracle.  With "device" (one rank)
         the slab uses the device form of the callbacks.
"""
import ctypes
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def slab_range(rank, world, ntau):
    """Slices of a rank: contiguous, sizes differing by at most one."""
    return rank * ntau // world, (rank + 1) * ntau // world


def comm_check(out):
    import torch
    import torch.distributed as dist
    from paper_1007_3432_gb300.binding import TorchDistComm
    dist.init_process_group("gloo")
    r, w = dist.get_rank(), dist.get_world_size()
    comm = TorchDistComm()
    send = torch.full((5,), float(r), dtype=torch.float64)
    recv = torch.empty(5, dtype=torch.float64)
    comm.exchange_host(+1, send, recv)          # from the previous rank
    assert torch.all(recv == float((r - 1) % w)), recv
    comm.exchange_host(-1, send, recv)          # from the next rank
    assert torch.all(recv == float((r + 1) % w)), recv
    v = torch.tensor([1.0, float(r)], dtype=torch.float64)
    comm.allreduce_host(v)
    assert v[0] == w and v[1] == w * (w - 1) / 2, v
    # the C-callable callbacks on host buffers, as the library calls them
    c = comm.c_callbacks()
    sbuf = (ctypes.c_double * 3)(r, r, r)
    rbuf = (ctypes.c_double * 3)()
    assert c.exchange(None, +1, ctypes.addressof(sbuf), ctypes.addressof(rbuf), 24) == 0
    assert list(rbuf) == [float((r - 1) % w)] * 3, list(rbuf)
    vals = (ctypes.c_double * 2)(2.0, float(r))
    assert c.allreduce_sum(None, vals, 2) == 0
    assert list(vals) == [2.0 * w, w * (w - 1) / 2.0], list(vals)
    open(os.path.join(out, "comm_ok_%d" % r), "w").write("ok")
    dist.destroy_process_group()


def gpu_run(out, d, nx, ntau, device=False):
    import torch
    import torch.distributed as dist
    import workloads
    import paper_1007_3432_gb300 as pkg
    from paper_1007_3432_gb300.binding import HH_OP_M, HH_OP_MT, HH_OP_MTM, Slab
    dist.init_process_group("gloo")
    r, w = dist.get_rank(), dist.get_world_size()
    torch.cuda.set_device(0)
    pkg.load()
    V = nx ** d
    n = V * ntau
    t0, t1 = slab_range(r, w, ntau)
    sigma = workloads.sigma_field(n, seed=700 + nx + ntau)
    x = workloads.source(n, seed=701)
    b = workloads.source(n, seed=702)
    part = slice(V * t0, V * t1)
    res = {"range": np.array([t0, t1])}
    # the device form on a stream of its own (its iterations replay as a CUDA graph)
    stream = torch.cuda.Stream() if device else None
    with Slab(d, nx, ntau, t0, t1, device_comm=device, stream=stream) as s:
        s.set_field(sigma[part].copy())
        xd = torch.from_numpy(x[part].copy()).cuda()
        y = torch.empty_like(xd)
        for name, op in (("M", HH_OP_M), ("MT", HH_OP_MT), ("MTM", HH_OP_MTM)):
            s.apply(op, xd, y)
            res[name] = y.cpu().numpy()
        bd = torch.from_numpy(b[part].copy()).cuda()
        xs = torch.zeros_like(bd)
        if stream is not None:
            stream.wait_stream(torch.cuda.current_stream())
        rc, info = s.solve(bd, xs)
        if stream is not None:
            torch.cuda.current_stream().wait_stream(stream)
        res["x"] = xs.cpu().numpy()
        res["info"] = np.array([rc, info["iterations"], info["true_relres"], info["converged"]])
    np.savez(os.path.join(out, "rank%d.npz" % r), **res)
    dist.destroy_process_group()


if __name__ == "__main__":
    if sys.argv[1] == "comm":
        comm_check(sys.argv[2])
    else:
        gpu_run(sys.argv[2], int(sys.argv[3]), int(sys.argv[4]), int(sys.argv[5]),
                device=len(sys.argv) > 6 and sys.argv[6] == "device")
