"""The two exchanges of the K-partitioned iteration across ranks (no GPU): world size 2 over gloo.

Eq. (11) sums over the samples, so a plan split into K-slices (one per rank) exchanges the
minimum cost with its global index and the finite count, then the sums of the softmin
normalisers and of the weighted noise.  The rank collectives must give what the one-process
combination gives: the same minimum record (ties to the lowest global index) and the same
binary64 totals up to the order of the additions.
"""
import json
import math
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2308_01654_gb300 import partition  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _records(case):
    """Per-rank (s_min, global argmin, n_finite) and (eta, du[3][2]) of a synthetic split."""
    rng = np.random.default_rng(5)
    sums = [(float(rng.uniform(1.0, 50.0)), rng.normal(size=(3, 2))) for _ in range(2)]
    if case == "distinct":
        mins = [(12.5, 17, 2048), (11.25, 2049, 1000)]
    elif case == "tie":                       # equal minima: the lower global index wins
        mins = [(3.0, 2040, 2048), (3.0, 2048, 512)]
    else:                                     # rank 0 has no finite cost
        mins = [(math.inf, -1, 0), (7.5, 4100, 300)]
    return mins, sums


def _rank_main(rank, world, port, out_dir, case):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2308_01654_gb300 import partition as part
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mins, sums = _records(case)
        m = part.allreduce_minima(*mins[rank])
        eta, du = part.allreduce_sums(*sums[rank])
        dist.barrier()
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"min": list(m), "eta": eta, "du": du.tolist()}, f)


@pytest.mark.parametrize("case", ["distinct", "tie", "empty_rank"])
def test_rank_exchanges_equal_the_one_process_combination(tmp_path, case):
    torch_mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    torch_mp.start_processes(_rank_main, args=(2, port, str(tmp_path), case), nprocs=2, join=True,
                             start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{i}.json")) for i in range(2)]
    mins, sums = _records(case)
    exp_min = partition.combine_minima(mins)
    exp_eta, exp_du = partition.combine_sums(sums)
    for q in r:
        assert tuple(q["min"]) == exp_min
        assert q["eta"] == pytest.approx(exp_eta, rel=1e-15)
        np.testing.assert_allclose(np.array(q["du"]), exp_du, rtol=1e-15, atol=1e-15)
    assert r[0] == r[1]


def test_one_process_combination():
    assert partition.combine_minima([(2.0, 5, 3), (1.0, 9, 4), (1.0, 7, 1)]) == (1.0, 7, 8)
    assert partition.combine_minima([(math.inf, -1, 0), (math.inf, -1, 0)]) == (math.inf, -1, 0)
    eta, du = partition.combine_sums([(1.5, np.ones((2, 2))), (2.5, 2 * np.ones((2, 2)))])
    assert eta == 4.0 and np.all(du == 3.0)
    assert partition.slice_offsets([2048, 2048, 100]) == [0, 2048, 4096]
