"""Multi-process (world size 2, gloo, CPU) tests of the multi-GPU host logic.

* replicas: per-rank seeds differ, the job time is the slowest rank's and the
  job rate counts every rank's units;
* channel sharding: per-rank partial averages over disjoint channel ranges,
  combined by an all-reduce, equal the full-band average (FP64 oracle);
* the ionospheric offset exchange: per-rank six numbers per source over
  disjoint channel ranges, summed by an all-reduce, equal the full band's;
* the channel-shard cadence driver (replicas.run_sharded_cadence with
  replicas.sum_over_ranks): two ranks, each peeling its half of the band with
  the oracle's steps and summing the partial averages before every solve,
  reproduce the oracle's whole-band peel.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(rank, world, port, fn, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, fn(rank, world)))
    finally:
        dist.destroy_process_group()


def _spawn(fn, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_run, args=(r, world, port, fn, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def _replica_logic(rank, world):
    from paper_1003_5575_gb300 import replicas
    assert replicas.world() == (rank, world)
    seed = replicas.rank_seed(100303, rank)
    t_max = replicas.max_over_ranks(1.0 + rank)          # rank 1 is slower
    replicas.barrier()
    return seed, t_max, replicas.job_rate(10.0, t_max, world)


def test_replicas_seed_time_and_rate():
    out = _spawn(_replica_logic)
    assert out[0][0] != out[1][0]
    assert out[0][1] == out[1][1] == 2.0                 # the slowest rank's time
    assert out[0][2] == pytest.approx(2 * 10.0 / 2.0)


def _sharded_average(rank, world):
    import oracle
    from paper_1003_5575_gb300 import replicas
    from synth import Cadence
    cad = Cadence(10, 24, 3, 2, seed=321)
    V = oracle.simulate(cad)
    l, m, _ = cad.sources()[0]
    full = oracle.rotate_average(cad.uvw(), cad.freqs(), V, l, m)
    lo, hi = rank * cad.n_chan // world, (rank + 1) * cad.n_chan // world
    part = oracle.rotate_average(cad.uvw(), cad.freqs()[lo:hi], V[:, :, lo:hi], l, m)
    comb = replicas.combine_partial_averages(torch.from_numpy(part.copy()), (hi - lo) * cad.n_time,
                                             cad.n_chan * cad.n_time)
    return np.abs(comb.numpy() - full).max(), np.abs(full).max()


def test_channel_sharded_partial_averages_allreduce_to_full_average():
    out = _spawn(_sharded_average)
    for err, scale in out.values():
        assert err <= 1e-13 * scale


def _sharded_offsets(rank, world):
    import oracle
    from paper_1003_5575_gb300 import replicas
    from synth import Cadence
    cad = Cadence(8, 20, 2, 3, pos_sigma_rad=2e-4, seed=322)
    V = oracle.simulate(cad.with_(pos_sigma_rad=0.0))
    src, J, f = cad.perturbed_sources(), cad.jones(), cad.freqs()
    full, off_full = oracle.offsets(cad.uvw(), f, V, src, J, alpha=2.0, nu_ref=150e6)
    lo, hi = rank * cad.n_chan // world, (rank + 1) * cad.n_chan // world
    part, _ = oracle.offsets(cad.uvw(), f[lo:hi], V[:, :, lo:hi], src, J, alpha=2.0, nu_ref=150e6)
    comb = replicas.combine_offset_statistics(torch.from_numpy(part.copy())).numpy()
    return np.abs(comb - full).max(), np.abs(full).max()


def test_offset_statistics_allreduce_to_full_band():
    out = _spawn(_sharded_offsets)
    for err, scale in out.values():
        assert err <= 1e-12 * scale


def _sharded_peel(rank, world):
    import oracle
    from paper_1003_5575_gb300 import replicas
    from synth import Cadence
    cad = Cadence(10, 24, 3, 4, seed=323)
    uvw, f, src = cad.uvw(), cad.freqs(), cad.sources()
    V = oracle.simulate(cad)
    R_ref, J_ref, _ = oracle.peel(uvw, f, V, src)
    lo, hi = rank * cad.n_chan // world, (rank + 1) * cad.n_chan // world
    w = (hi - lo) / cad.n_chan                      # this rank's share of the band's samples
    state = {"R": V[:, :, lo:hi].copy(), "k": 0, "J": []}

    def partials():                                 # this rank's part of the band's average
        l, m, _ = src[state["k"]]
        state["avg"] = torch.from_numpy(w * oracle.rotate_average(uvw, f[lo:hi], state["R"], l, m))
        return state["avg"]

    def step():                                     # solve from the summed average, subtract locally
        k = state["k"]
        l, m, S = src[k]
        J, _, _ = oracle.als(state["avg"].numpy(), S, cad.n_ant)
        state["J"].append(J)
        state["R"] = oracle.subtract(uvw, f[lo:hi], state["R"], l, m, S, J)
        state["k"] += 1
        return 1 if state["k"] < len(src) else 0

    n = replicas.run_sharded_cadence(lambda: None, partials, step, replicas.sum_over_ranks)
    err_r = np.abs(state["R"] - R_ref[:, :, lo:hi]).max() / np.abs(V).max()
    err_j = max(np.abs(state["J"][k] - J_ref[k]).max() for k in range(len(src)))
    return n, err_r, err_j


def test_channel_shard_cadence_driver_reproduces_whole_band_peel():
    out = _spawn(_sharded_peel)
    for n, err_r, err_j in out.values():
        assert n == 4
        assert err_r <= 1e-12 and err_j <= 1e-10
