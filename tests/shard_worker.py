"""One rank of a row-sharded solve, run as its own process by tests/test_shard.py and
tests/test_gpu_sharded.py (environment: RANK, WORLD_SIZE, MASTER_ADDR, MASTER_PORT).

    python tests/shard_worker.py reduce OUT.npz            # host reduction only (CPU)
    python tests/shard_worker.py solve OUT.npz m n k p q dtype seed   # rsvd_sharded on cuda:0
    python tests/shard_worker.py leave OUT.npz m n k p q dtype seed   # rank 1 leaves before solving
"""
import ctypes
import datetime
import os
import sys

import numpy as np
import torch
import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import paper_1906_12085_gb300 as g  # noqa: E402
from paper_1906_12085_gb300 import shard  # noqa: E402


def matrix(m, n, seed):
    import synth
    sig = synth.spectrum_harmonic_noise(n, seed + 2)
    A = synth.prescribed(m, n, sig, seed, seed + 1)
    return A + torch.linspace(-1.0, 2.0, n, dtype=torch.float64).unsqueeze(0)


def main():
    mode, out = sys.argv[1], sys.argv[2]
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    if mode == "reduce":
        fn = g.allreduce_callback(shard.dist_allreduce())
        buf = (np.arange(7, dtype=np.float64) + 1.0) * (rank + 1)
        rc = fn(buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), buf.size, None)

        def boom(_):
            raise RuntimeError("reduction failed")
        bad = g.allreduce_callback(boom)
        one = np.zeros(1)
        rc_bad = bad(one.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1, None)
        np.savez(out, buf=buf, rc=rc, rc_bad=rc_bad, r0r1=np.array(shard.row_block(20011, world, rank)))
        dist.barrier()
        dist.destroy_process_group()
        return
    m, n, k, p, q = (int(x) for x in sys.argv[3:8])
    dtype, seed = sys.argv[8], int(sys.argv[9])
    r0, r1 = shard.row_block(m, world, rank)
    A = matrix(m, n, seed)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    gdt = g.RSVD_F32 if dtype == "f32" else g.RSVD_F64
    import synth
    Om = synth.gaussian(n, k + p, seed=seed + 3, dtype=tdt).to("cuda")
    Ar = A[r0:r1].to(device="cuda", dtype=tdt).contiguous()
    S = torch.zeros(k, dtype=torch.float64, device="cuda")
    U = torch.zeros(r1 - r0, k, dtype=tdt, device="cuda")
    V = torch.zeros(n, k, dtype=tdt, device="cuda")
    if mode == "leave":
        dist.barrier()
        if rank == 1:   # leaves between steps: nothing of it is in flight
            os._exit(0)
    with g.rsvd_plan_create(r1 - r0, n, k, p, q, gdt) as plan:
        st = g.rsvd_sharded(plan, m, Ar, Om, S, U, V, shard.dist_allreduce())
        sync = g.rsvd_plan_sync(plan)
        fro2 = g.rsvd_plan_fro2(plan) if st == g.RSVD_OK else float("nan")
    torch.cuda.synchronize()
    np.savez(out, st=st, sync=sync, S=S.cpu().numpy(), U=U.double().cpu().numpy(), V=V.double().cpu().numpy(),
             fro2=fro2, r0=r0, r1=r1)
    if mode != "leave":
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
