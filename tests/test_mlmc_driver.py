"""Host logic of the adaptive MLMC driver (section 3) with a synthetic
sampler, the cross-rank statistics merge on two gloo ranks, and (GPU) the
driver's estimator against the oracle's on the same samples."""
import math
import os

import numpy as np
import pytest

from oracle import mlmc as OM
from paper_2403_17018_gb300 import mlmc as M


class FakeSampler:
    """g_l - g_{l-1} ~ N(a 2^-l, v 4^-l) per QoI, cost 8^l per pair; sample
    i of level l is a fixed function of (l, i) like the real xi streams."""

    def __init__(self, a=0.3, v=0.04):
        self.a, self.v = a, v
        self.calls = []

    def draw(self, level, first, count):
        out_f, out_d = [], []
        for i in range(first, first + count):
            rng = np.random.default_rng(level * 1_000_003 + i)
            d = self.a * 2.0 ** -level + math.sqrt(self.v * 4.0 ** -level) * rng.standard_normal(M.NQ)
            out_d.append(d)
            out_f.append(d + 1.0)
        return np.array(out_f), np.array(out_d)

    def batch(self, level, first, count):
        self.calls.append((level, first, count))
        gf, gd = self.draw(level, first, count)
        st = OM.level_stats(gf, gf - gd)
        n = count
        return (n, st["mean_f"], st["var_f"] * (n - 1), st["mean_d"], st["var_d"] * (n - 1),
                8.0 ** level * count * 1e-3, 0)


def test_allocation_matches_eq_m_ell_and_meets_variance_budget():
    s = FakeSampler()
    eps = 0.01
    res = M.run(s, 3, eps, qois=(0, 1), pilot=[32, 16, 8, 8])
    V = np.array(res["V_l"])[:, :2]
    cost = np.array(res["seconds_per_pair"])
    m = np.max(np.stack([M.allocate(V[:, k], cost, eps) for k in range(2)]), axis=0)
    assert all(res["n"][l] >= m[l] for l in range(4))
    # independent formula from the oracle module
    mo = np.max(np.stack([OM.allocation(V[:, k], cost, eps) for k in range(2)]), axis=0)
    assert list(m) == list(mo)
    assert max(res["var_Y"][:2]) <= eps**2 / 2 * (1 + 1e-12)
    # telescoping: the estimate is the sum of level means
    assert np.allclose(res["estimate"], np.sum(res["mean_l"], axis=0), atol=1e-15)


def test_estimate_is_within_its_error_of_the_truth():
    s = FakeSampler()
    eps = 0.005
    res = M.run(s, 4, eps, qois=(0,))
    truth = sum(s.a * 2.0 ** -l for l in range(5))
    err = abs(res["estimate"][0] - truth)
    assert err <= 4 * math.sqrt(res["var_Y"][0]) + 1e-12


def test_resume_draws_only_new_samples():
    s = FakeSampler()
    r1 = M.run(s, 2, 0.05, qois=(0,))
    s2 = FakeSampler()
    r2 = M.run(s2, 2, 0.02, qois=(0,), state=r1["state"])
    first_new = {l: r1["state"][l]["drawn"] for l in range(3)}
    for (l, first, count) in s2.calls:
        assert first >= first_new[l]
    full = M.run(FakeSampler(), 2, 0.02, qois=(0,), pilot=r2["n"])
    assert r2["n"] == full["n"] or all(a >= b for a, b in zip(r2["n"], full["n"]))


def _rank_main(rank, world, port, result_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)

    class Sliced(FakeSampler):
        def batch(self, level, first, count):
            lo = first + (count * rank) // world
            hi = first + (count * (rank + 1)) // world
            return super().batch(level, lo, hi - lo)

    res = M.run(Sliced(), 2, 0.02, qois=(0, 1), dist=dist)
    if rank == 0:
        np.save(result_path, np.array(res["estimate"] + res["var_Y"] + res["n"], dtype=float))
    dist.destroy_process_group()


def test_two_gloo_ranks_match_one_rank(tmp_path):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        port = sck.getsockname()[1]
    out = str(tmp_path / "r.npy")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, start_method="spawn")
    got = np.load(out)
    ref = M.run(FakeSampler(), 2, 0.02, qois=(0, 1))
    want = np.array(ref["estimate"] + ref["var_Y"] + ref["n"], dtype=float)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-15)


@pytest.mark.gpu
def test_gpu_estimator_matches_oracle_on_the_same_samples():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_helpers import oracle_solve, tight_config
    from paper_2403_17018_gb300.inputs import xi_batch
    cfg = tight_config(nlevels=2)
    sampler = M.GpuSampler(cfg)
    res = M.run(sampler, 1, 10.0, pilot=[8, 4], max_batch=[8, 4])
    assert res["n"] == [8, 4] and res["failed"] == 0
    g0 = np.array([oracle_solve(cfg, 0, x)[2] for x in xi_batch(0, 0, 8)])
    x1 = xi_batch(1, 0, 4)
    d1 = np.array([oracle_solve(cfg, 1, x)[2] - oracle_solve(cfg, 0, x)[2] for x in x1])
    Y = g0.mean(0) + d1.mean(0)
    var = g0.var(0, ddof=1) / 8 + d1.var(0, ddof=1) / 4
    assert np.allclose(res["estimate"], Y, rtol=1e-9, atol=1e-10)
    assert np.allclose(res["var_Y"], var, rtol=1e-6, atol=1e-16)


def test_a_level_without_valid_samples_stops_the_run():
    class Failing(FakeSampler):
        def batch(self, level, first, count):
            if level == 2:
                return (0, np.zeros(M.NQ), np.zeros(M.NQ), np.zeros(M.NQ), np.zeros(M.NQ), 1.0, count)
            return super().batch(level, first, count)

    with pytest.raises(RuntimeError, match="level"):
        M.run(Failing(), 2, 0.01, qois=(0,))


def test_concurrent_waves_give_the_sequential_result():
    """With a sampler that runs several levels at once, every level still
    merges its batches in the same order, so the result is identical."""
    class Multi(FakeSampler):
        def batches(self, reqs):
            return [self.batch(*r) for r in reqs]

    seq = M.run(FakeSampler(), 3, 0.01, qois=(0, 1), max_batch=[64, 16, 8, 4], concurrent=False)
    con = M.run(Multi(), 3, 0.01, qois=(0, 1), max_batch=[64, 16, 8, 4], concurrent=True)
    for k in ("estimate", "var_Y", "n", "mean_l", "V_l"):
        assert con[k] == seq[k], k


@pytest.mark.parametrize("eps", [2e-2, 5e-3, 1e-3])
def test_adaptive_level_count_matches_the_bias_model(eps):
    """With corrections E Y_l = a 2^-l and (almost) no noise, the driver adds
    levels until Eq. num_levels is met: the finest level is the smallest L
    whose tail bias a 2^-L is at most eps / sqrt(2), as the oracle's
    weak-error fit and level formula give for the same level means."""
    s = FakeSampler(v=1e-20)
    res = M.run(s, 12, eps, qois=(0,), adaptive_levels=True, L_start=2)
    L = res["levels"] - 1
    brute = next(k for k in range(40) if s.a * 2.0 ** -k <= eps / math.sqrt(2.0))
    assert L == max(brute, 2)
    alpha, c1 = OM.weak_error_constants(list(range(1, L + 1)), [m[0] for m in res["mean_l"][1:]])
    assert OM.num_levels(eps, 1.0, c1, alpha) == brute
    # levels were added one at a time, each decision from the levels so far
    assert [c["levels_fitted"] for c in res["level_choice"]][:L - 2] == list(range(3, L + 1))


def test_relative_tolerance_scales_by_level_zero_mean():
    """relative=True: eps is relative to E0 = |E g_0| (Eq. scaled_m_l_S): the
    run ends with Var Y within (eps E0)^2 / 2, E0 the level-0 mean of g, and
    allocates Eq. M_ell with eps E0."""
    s = FakeSampler()
    eps = 0.01
    res = M.run(s, 3, eps, qois=(0,), relative=True, pilot=[32, 16, 8, 8])
    E0 = abs(res["state"][0]["mean_f"][0])
    assert res["var_Y"][0] <= (eps * E0) ** 2 / 2 * (1 + 1e-12)
    V = np.array(res["V_l"])[:, 0]
    m = OM.allocation(V, np.array(res["seconds_per_pair"]), eps * E0)
    assert all(n >= k for n, k in zip(res["n"], m))


def test_adaptive_run_resumes_from_its_state():
    """Resuming an adaptive-level run at a tighter eps keeps every drawn
    sample, draws only new indices, and may add finer levels; the result
    equals a fresh adaptive run whose pilots are the first run's counts."""
    s1 = FakeSampler(v=1e-20)
    r1 = M.run(s1, 10, 2e-2, qois=(0,), adaptive_levels=True)
    s2 = FakeSampler(v=1e-20)
    r2 = M.run(s2, 10, 2e-3, qois=(0,), adaptive_levels=True, state=r1["state"])
    drawn = {l: r1["state"][l]["drawn"] for l in range(len(r1["state"]))}
    for (l, first, count) in s2.calls:
        assert first >= drawn.get(l, 0)
    assert r2["levels"] >= r1["levels"]
    brute = next(k for k in range(40) if s2.a * 2.0 ** -k <= 2e-3 / math.sqrt(2.0))
    assert r2["levels"] - 1 == brute
