"""Host side of the row-sharded solve (no GPU): the row-block partition and the reduction
callback over torch.distributed, with two gloo ranks as separate processes."""
import numpy as np
import pytest

from paper_1906_12085_gb300 import shard
from shard_ranks import run_ranks


@pytest.mark.parametrize("world", [1, 2, 3, 7, 8])
def test_row_block_partition(world):
    for m in (0, 1, 7, 8, 20011, 1 << 20):
        blocks = [shard.row_block(m, world, r) for r in range(world)]
        assert blocks[0][0] == 0 and blocks[-1][1] == m
        for (a0, a1), (b0, b1) in zip(blocks, blocks[1:]):
            assert a1 == b0
        sizes = [b - a for a, b in blocks]
        assert max(sizes) - min(sizes) <= (0 if m % world == 0 else 1)
        assert sizes == sorted(sizes, reverse=True)


def test_row_block_rejects_bad_arguments():
    for args in ((10, 0, 0), (10, 2, 2), (10, 2, -1), (-1, 2, 0)):
        with pytest.raises(ValueError):
            shard.row_block(*args)


def test_reduction_callback_over_two_gloo_ranks(tmp_path):
    procs, outs, logs = run_ranks(2, ["reduce"], tmp_path)
    for p, log in zip(procs, logs):
        assert p.returncode == 0, log
    r = [np.load(o) for o in outs]
    expect = (np.arange(7, dtype=np.float64) + 1.0) * 3.0   # rank 0 holds 1x, rank 1 2x
    for x in r:
        assert int(x["rc"]) == 0 and int(x["rc_bad"]) == 1
        assert np.array_equal(x["buf"], expect)
    assert tuple(r[0]["r0r1"]) == (0, 10006) and tuple(r[1]["r0r1"]) == (10006, 20011)
