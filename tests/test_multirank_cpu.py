"""World-size-2 gloo test of the multi-rank path (CPU only).

Each rank runs its own disorder sample (here with the oracle standing in for
the GPU work), the only collective is the MAX reduction of the elapsed time,
and each rank's result equals the same sample run alone.
"""
import json
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

L = 6
SWEEPS = 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_sample(sample):
    import oracle
    from paper_1006_2566_gb300 import inputs

    J = inputs.round_to_f32(inputs.gaussian_couplings(L, seed=3, sample=sample))
    s = oracle.init_spins(L, 3, sample)
    sch = oracle.Schedule(kind=oracle.HB, beta=1 / 0.7, n_or=2, energy_every=1)
    _, elog = oracle.sweeps(L, J, s, sch, oracle.key(3, sample), SWEEPS)
    return float(np.sum(J)), list(map(float, elog))


def _worker(rank, world, port, outdir):
    import time

    from paper_1006_2566_gb300 import dist as hdist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = hdist.env()
    sample = hdist.rank_sample(r)
    t0 = time.perf_counter()
    jsum, elog = _run_sample(sample)
    elapsed = time.perf_counter() - t0 + 0.01 * r  # make the ranks' times differ
    tmax = hdist.max_over_ranks(elapsed)
    gathered = [None] * world
    dist.all_gather_object(gathered, elapsed)
    with open(os.path.join(outdir, f"rank{r}.json"), "w") as f:
        json.dump({"world": w, "rank": r, "local": lr, "sample": sample, "jsum": jsum, "elog": elog,
                   "elapsed": elapsed, "tmax": tmax, "all": gathered,
                   "thr": hdist.job_throughput(SWEEPS * L ** 3, w, tmax)}, f)
    dist.destroy_process_group()


def test_two_ranks_run_independent_samples_and_reduce_time():
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(world, _free_port(), d), nprocs=world, start_method="spawn")
        res = [json.load(open(os.path.join(d, f"rank{r}.json"))) for r in range(world)]
    assert [r["rank"] for r in res] == [0, 1] and all(r["world"] == 2 for r in res)
    assert res[0]["sample"] != res[1]["sample"]
    assert res[0]["jsum"] != res[1]["jsum"]  # different couplings per rank
    for r in res:
        assert r["tmax"] == max(r["all"])
        assert r["thr"] == pytest.approx(SWEEPS * L ** 3 * 2 / r["tmax"])
        jsum, elog = _run_sample(r["sample"])  # the same sample alone
        assert jsum == r["jsum"] and elog == r["elog"]


def test_single_process_helpers():
    from paper_1006_2566_gb300 import dist as hdist

    assert hdist.max_over_ranks(3.5) == 3.5
    assert hdist.rank_sample(3, base_sample=10) == 13
    assert hdist.job_throughput(100, 4, 2.0) == 200
    with pytest.raises(ValueError):
        hdist.job_throughput(1, 1, 0.0)
