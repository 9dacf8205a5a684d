"""Batched small solves (rsvd_batch_*): several randomized PCA problems of the
same l and q in lockstep, the small dense steps batched into single launches.
Each problem runs the same kernels as a single rsvd() call, so its results are
compared bit for bit with the problem solved alone, and one of them with the
FP64 oracle (tolerance of the float32 path: 1e-5 sigma_1)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1906_12085_gb300 as g
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_12085_gb300 import build
    build.build()


# (m, n, k, p): l = k + p = 28 for all, so they share a batch
SHAPES = [(5000, 300, 20, 8), (3001, 128, 20, 8), (12000, 64, 12, 16), (4096, 1000, 24, 4), (777, 40, 28, 0)]
Q = 2


def _problem(i, m, n, k, p):
    sig = synth.spectrum_power(n, 1.0 + 0.1 * i)
    A = synth.prescribed(m, n, sig, 500 + i, 600 + i) + torch.linspace(-1.0, 2.0, n, dtype=torch.float64)
    Om = synth.gaussian(n, k + p, seed=700 + i, dtype=torch.float32)
    return A.float(), Om


def _bufs(m, n, k, dev):
    return (torch.zeros(k, dtype=torch.float64, device=dev), torch.zeros(m, k, device=dev),
            torch.zeros(n, k, device=dev))


def _alone(A, Om, k, p):
    dev = torch.device("cuda")
    m, n = A.shape
    Ad, Od = A.to(dev), Om.to(dev)
    S, U, V = _bufs(m, n, k, dev)
    with g.rsvd_plan_create(m, n, k, p, Q, g.RSVD_F32) as plan:
        g.check(g.rsvd(plan, Ad, None, Od, S, U, V))
        st = g.rsvd_plan_sync(plan)
        stK, K = g.pca_threshold(plan, 0.9)
    torch.cuda.synchronize()
    return st, K, S.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy()


def _batched(probs, batch_stream, plan_streams, workspace=False, runs=1):
    dev = torch.device("cuda")
    plans, keep = [], []
    A, Om, S, U, V = [], [], [], [], []
    for (Ah, Oh, k, p), ps in zip(probs, plan_streams):
        m, n = Ah.shape
        if workspace:
            st, nb = g.rsvd_workspace_query(m, n, k, p, Q)
            g.check(st)
            ws = torch.empty(nb, dtype=torch.uint8, device=dev)
            plans.append(g.rsvd_plan_create_in(m, n, k, p, Q, g.RSVD_F32, ps, ws))
        else:
            plans.append(g.rsvd_plan_create(m, n, k, p, Q, g.RSVD_F32, ps))
        A.append(Ah.to(dev))
        Om.append(Oh.to(dev))
        s, u, v = _bufs(m, n, k, dev)
        S.append(s)
        U.append(u)
        V.append(v)
    torch.cuda.synchronize()
    out = []
    with g.rsvd_batch_create(plans, batch_stream) as b:
        for _ in range(runs):
            g.check(g.rsvd_batch_run(b, A, Om, S, U, V), "rsvd_batch_run")
            st, sts = g.rsvd_batch_sync(b)
            Ks = [g.pca_threshold(P, 0.9)[1] for P in plans]
            out.append((st, sts, Ks, [x.cpu().numpy() for x in S], [x.cpu().numpy() for x in U],
                        [x.cpu().numpy() for x in V]))
    for P in plans:
        P.close()
    return out


def _probs():
    return [(*_problem(i, m, n, k, p), k, p) for i, (m, n, k, p) in enumerate(SHAPES)]


def test_batch_equals_alone_bitwise_and_replays():
    probs = _probs()
    alone = [_alone(A, Om, k, p) for A, Om, k, p in probs]
    streams = [torch.cuda.Stream() for _ in probs]
    runs = _batched(probs, torch.cuda.Stream(), streams, runs=2)
    for st, sts, Ks, S, U, V in runs:          # first run captures the graph, the second replays it
        assert st == g.RSVD_OK and sts == [g.RSVD_OK] * len(probs)
        for i, (a_st, a_K, a_S, a_U, a_V) in enumerate(alone):
            assert Ks[i] == a_K
            assert np.array_equal(S[i], a_S), i
            assert np.array_equal(U[i], a_U), i
            assert np.array_equal(V[i], a_V), i


def test_batch_matches_oracle():
    A, Om, k, p = _probs()[0]
    (st, sts, Ks, S, U, V), = _batched([(A, Om, k, p)], torch.cuda.Stream(), [torch.cuda.Stream()])
    Ac, mu, fro2 = oracle.center(A.double())
    s, Uo, Vo = oracle.rsvd(Ac, Om.double(), q=Q, k=k)
    assert np.abs(S[0] - s).max() <= 1e-5 * s[0]


def test_batch_on_legacy_stream_and_caller_workspace():
    """Direct launches (no graph) and plans carved from caller-owned workspace give the same bits."""
    probs = _probs()[:3]
    alone = [_alone(A, Om, k, p) for A, Om, k, p in probs]
    (st, sts, Ks, S, U, V), = _batched(probs, 0, [0, 0, 0], workspace=True)
    assert st == g.RSVD_OK
    for i, (a_st, a_K, a_S, a_U, a_V) in enumerate(alone):
        assert np.array_equal(S[i], a_S) and np.array_equal(U[i], a_U) and np.array_equal(V[i], a_V)


def test_batch_rejects_mixed_l_and_duplicates():
    dev = torch.device("cuda")
    p1 = g.rsvd_plan_create(1000, 64, 8, 4, Q, g.RSVD_F32)
    p2 = g.rsvd_plan_create(1000, 64, 8, 8, Q, g.RSVD_F32)
    with pytest.raises(g.RsvdError):
        g.rsvd_batch_create([p1, p2])
    with pytest.raises(g.RsvdError):
        g.rsvd_batch_create([p1, p1])
    p1.close()
    p2.close()
    # l > 128: the batched small kernels keep l x l blocks in shared memory
    p3 = g.rsvd_plan_create(2000, 300, 136, 8, Q, g.RSVD_F32)
    with pytest.raises(g.RsvdError) as e:
        g.rsvd_batch_create([p3])
    assert e.value.status == g.RSVD_ERR_UNSUPPORTED
    p3.close()
    del dev
