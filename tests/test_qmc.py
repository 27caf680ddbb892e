"""Halton points, sample quantiles and exceedance statistics of the QMC runs
(section 4, tests A1-A3), and (GPU) a small QMC run against the oracle."""
import numpy as np
import pytest

from oracle import qmc as OQ
from paper_2403_17018_gb300.inputs import halton, radical_inverse, xi_halton
from paper_2403_17018_gb300.qmc import sample_quantiles


def test_radical_inverse_textbook_values():
    """van der Corput: base 2 gives 0, 1/2, 1/4, 3/4, 1/8, 5/8, ...; base 3
    gives 0, 1/3, 2/3, 1/9, 4/9, 7/9, 2/9, ..."""
    assert radical_inverse(np.arange(8), 2).tolist() == [0, .5, .25, .75, .125, .625, .375, .875]
    b3 = [0, 1 / 3, 2 / 3, 1 / 9, 4 / 9, 7 / 9, 2 / 9, 5 / 9, 8 / 9]
    assert np.allclose(radical_inverse(np.arange(9), 3), b3, rtol=0, atol=1e-15)
    # 1234 = 1*5^4 + 4*5^3 + 4*5^2 + 1*5 + 4: digits 4, 1, 4, 4, 1 mirrored
    assert radical_inverse(np.array([1234]), 5)[0] == pytest.approx(
        sum(d * 5.0 ** -(k + 1) for k, d in enumerate([4, 1, 4, 4, 1])), abs=1e-15)


@pytest.mark.parametrize("base,k", [(2, 10), (3, 6), (5, 4), (13, 2)])
def test_first_b_to_the_k_points_are_equidistributed(base, k):
    """The first b^k radical inverses in base b are exactly {j / b^k}."""
    n = base ** k
    u = np.sort(radical_inverse(np.arange(n), base))
    assert np.allclose(u, np.arange(n) / n, rtol=0, atol=1e-14)


def test_halton_dimensions_and_shift():
    u = halton(1, 100, 6)
    assert u.shape == (100, 6) and np.all((u >= 0) & (u < 1))
    assert np.array_equal(u[:, 1], radical_inverse(np.arange(1, 101), 3))
    a, b = halton(1, 50, 3, shift_seed=5), halton(1, 50, 3, shift_seed=5)
    assert np.array_equal(a, b)
    d = np.mod(a - halton(1, 50, 3), 1.0)     # one shift per coordinate
    assert np.allclose(d, d[0], atol=1e-12)
    xi = xi_halton(1, 10, 3)
    assert np.all((xi >= -1) & (xi < 1)) and np.allclose(xi, 2 * halton(1, 10, 3) - 1)


def test_oracle_quantile_closed_forms():
    """Definition 7 on a permutation of 0..n-1 gives (n-1) p; on {a, b},
    a + p (b - a); the median of an odd sample is its middle order statistic."""
    for n in (2, 5, 600):
        for p in (0.0, 0.025, 0.25, 0.5, 0.975, 1.0):
            assert OQ.quantile(np.random.default_rng(n).permutation(n), p) == \
                pytest.approx((n - 1) * p, abs=1e-12)
    assert OQ.quantile([3.0, 1.0], 0.25) == pytest.approx(1.5)
    assert OQ.quantile([5.0, -2.0, 9.0, 0.5, 7.0], 0.5) == 5.0


def test_driver_quantiles_match_the_oracle():
    rng = np.random.default_rng(1)
    probs = (0.025, 0.25, 0.5, 0.75, 0.975)
    for n in (1, 7, 600):
        x = rng.standard_normal((n, 3))
        got = sample_quantiles(x, probs)
        for i, p in enumerate(probs):
            for k in range(3):
                assert got[i, k] == pytest.approx(OQ.quantile(x[:, k], p), abs=1e-14)


def test_replicate_estimate_closed_form():
    m, se = OQ.replicate_estimate([[1.0], [3.0]])
    assert m[0] == 2.0 and se[0] == pytest.approx(1.0)


torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_exceedance_counts_are_exact():
    """mlmc_field_exceedance counts c > threshold per cell over valid
    samples, accumulated over batches: equal to numpy brute force."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_17018_gb300 import binding as hb
    ctx = hb.Context(hb.default_config(nlevels=2))
    rng = np.random.default_rng(3)
    c = rng.random((37, 64 * 32))
    c[5, :10] = 0.5                               # ties at the threshold do not count
    st = np.zeros(37, dtype=np.int32)
    st[[2, 30]] = 1
    count = torch.zeros(64 * 32, dtype=torch.int64, device="cuda")
    cd = torch.from_numpy(c).cuda()
    sd = torch.from_numpy(st).cuda()
    ctx.field_exceedance(1, cd[:20].contiguous(), sd[:20].contiguous(), 0.5, count)
    ctx.field_exceedance(1, cd[20:].contiguous(), sd[20:].contiguous(), 0.5, count)
    want = np.sum(c[st == 0] > 0.5, axis=0)
    assert np.array_equal(count.cpu().numpy(), want)
    with pytest.raises(hb.HenryError):
        ctx.field_exceedance(1, cd, sd, float("nan"), count)


@pytest.mark.gpu
def test_qmc_run_matches_the_oracle():
    """12 Halton points per replicate on level 0 in batches of 5 (ragged),
    two shifted replicates: the replicate means, the quantiles and the
    exceedance field agree with the oracle's solves of the same xi."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_helpers import oracle_solve, tight_config
    from paper_2403_17018_gb300 import binding as hb
    from paper_2403_17018_gb300 import qmc as Q
    cfg = tight_config(nlevels=1)
    ctx = hb.Context(cfg)
    res = Q.run(ctx, 0, 12, batch=5, replicates=2, thresholds=(0.3,))
    assert res["failed"] == 0
    qs, cs = [], []
    for r in range(2):
        xi = xi_halton(1, 12, 3, 2403017018 + 7919 * (r + 1))
        sol = [oracle_solve(cfg, 0, x) for x in xi]
        q = np.array([s[2] for s in sol])
        assert np.allclose(res["replicate_means"][r], q.mean(axis=0), rtol=1e-9, atol=1e-10)
        qs.append(q)
        cs.append(np.array([s[1] for s in sol]))
    q = np.concatenate(qs)
    for i, p in enumerate(res["quantile_probs"]):
        for k in range(q.shape[1]):
            assert res["quantiles"][i, k] == pytest.approx(OQ.quantile(q[:, k], p), rel=1e-9,
                                                           abs=1e-10)
    mean, se = OQ.replicate_estimate(res["replicate_means"])
    assert np.allclose(res["mean"], mean, rtol=1e-14) and np.allclose(res["std_error"], se,
                                                                       rtol=1e-12)
    c = np.concatenate(cs)
    assert res["n_field"] == c.shape[0]
    near = np.any(np.abs(c - 0.3) < 1e-8, axis=0)   # decisions the 1e-9 parity may flip
    want = np.sum(c > 0.3, axis=0)
    got = res["counts"][0]
    bad = np.argwhere((got != want) & ~near)
    assert len(bad) == 0, [(int(j), int(i), int(got[j, i]), int(want[j, i])) for j, i in bad[:8]]
    ex = OQ.exceedance(c, 0.3)
    assert np.array_equal(res["exceedance"][0][~near], ex[~near])


@pytest.mark.gpu
def test_qoi_series_matches_the_oracle_states():
    """henry_solve_series: the 22 QoIs after every 4th of the 24 level-0
    steps equal the oracle's QoIs of its states at those steps, and the last
    entry is the QoI vector at T; QMC quantiles over time come from them."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_helpers import oracle_grid, oracle_physics, tight_config
    from oracle import henry as H
    from paper_2403_17018_gb300 import binding as hb
    from paper_2403_17018_gb300 import qmc as Q
    cfg = tight_config(nlevels=1)
    ctx = hb.Context(cfg)
    xi = torch.from_numpy(xi_halton(1, 3, 3)).cuda()
    out = ctx.solve_series(0, xi, 4)
    assert out["series"].shape == (3, 6, hb.NQ)
    assert torch.equal(out["series"][:, -1], out["q"])
    g, ph = oracle_grid(cfg, 0), oracle_physics(cfg)
    V = (cfg.Lx / cfg.nx0) * (cfg.Ly / cfg.ny0)
    for b in range(3):
        r = H.solve(g, ph, xi[b].cpu().numpy(), keep_states=True)
        for k in range(6):
            c = r["states"][4 * (k + 1)][1]
            want = H.qoi(g, ph, r["fields"], c)
            got = out["series"][b, k].cpu().numpy()
            keep = np.arange(hb.NQ) != 6
            assert np.allclose(got[keep], want[keep], rtol=1e-9, atol=1e-9)
            assert abs(got[6] - want[6]) <= V * np.sum(np.abs(c - H.FRESH_C) <= 1e-9) + 1e-12
    res = Q.run(ctx, 0, 5, batch=3, series_every=6)
    assert res["series_steps"] == [6, 12, 18, 24]
    assert res["series_quantiles"].shape == (4, 5, hb.NQ)
    assert np.allclose(res["series_quantiles"][-1], res["quantiles"], rtol=0, atol=0)


class _FakeCtx:
    """Stand-in for a context on the CPU: q and c are fixed smooth functions
    of xi, and the statistics entry points are plain numpy Welford/Chan
    updates, so that the driver's host logic (sharding, merging) can run on
    gloo ranks without a GPU."""

    class _Info:
        ny, nx, nt = 4, 6, 12

    def level_info(self, level):
        return self._Info()

    def solve(self, level, xi, want_c=False):
        import torch
        x = xi.numpy()
        from paper_2403_17018_gb300 import binding as hb
        q = np.stack([np.sin(x[:, 0] * (k + 1)) + x[:, 1] * k + x[:, 2] ** 2 for k in range(hb.NQ)], 1)
        cells = np.arange(24)
        c = 0.5 + 0.4 * np.sin(x[:, :1] * 3 + cells[None, :] * 0.7 + x[:, 1:2])
        st = np.zeros(len(x), dtype=np.int32)
        st[np.abs(x[:, 2]) > 0.97] = 1                       # a few "failed" samples
        return {"q": torch.from_numpy(q), "c": torch.from_numpy(c.reshape(-1, 4, 6)),
                "status": torch.from_numpy(st)}

    def level_stats(self, level, q, qc, st, S):
        ok = st.numpy() == 0
        v = q.numpy()[ok]
        nb = len(v)
        if nb == 0:
            return
        mb = v.mean(0)
        m2b = ((v - mb) ** 2).sum(0)
        n = S.n + nb
        d = mb - np.array(S.mean_f[:])
        mean = np.array(S.mean_f[:]) + d * nb / n
        m2 = np.array(S.m2_f[:]) + m2b + d * d * S.n * nb / n
        S.n = n
        S.mean_f[:] = mean.tolist()
        S.m2_f[:] = m2.tolist()

    def field_stats(self, level, c, cc, st, acc):
        ok = st.numpy() == 0
        for row in c.numpy()[ok]:
            n = acc["n"] + 1
            d = row - acc["mean_f"].numpy()
            acc["mean_f"] += torch.from_numpy(d / n.numpy())
            acc["m2_f"] += torch.from_numpy(d * (row - acc["mean_f"].numpy()))
            acc["n"] += 1

    def field_exceedance(self, level, c, st, th, count):
        ok = st.numpy() == 0
        count += torch.from_numpy(np.sum(c.numpy()[ok] > th, axis=0))


def _qmc_rank(rank, world, port, out):
    import os
    import torch.distributed as dist
    from paper_2403_17018_gb300 import qmc as Q
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = Q.run(_FakeCtx(), 0, 23, batch=7, replicates=2, thresholds=(0.5,), rank=rank,
                world=world, dist=dist, device="cpu")
    if rank == 0:
        np.savez(out, mean=res["mean"], se=res["std_error"], quant=res["quantiles"],
                 var=res["var_field"], mf=res["mean_field"], ex=res["exceedance"][0],
                 failed=res["failed"])
    dist.destroy_process_group()


def test_qmc_on_two_gloo_ranks_equals_one_rank(tmp_path):
    """Each rank solves a disjoint slice of every batch; the merged replicate
    statistics, fields, exceedance and quantiles equal the one-rank run."""
    import socket
    import torch.multiprocessing as mp
    from paper_2403_17018_gb300 import qmc as Q
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "r.npz")
    mp.start_processes(_qmc_rank, args=(2, port, out), nprocs=2, start_method="spawn")
    got = np.load(out)
    ref = Q.run(_FakeCtx(), 0, 23, batch=7, replicates=2, thresholds=(0.5,), device="cpu")
    assert got["failed"] == ref["failed"] > 0
    assert np.allclose(got["mean"], ref["mean"], rtol=1e-13, atol=1e-15)
    assert np.allclose(got["se"], ref["std_error"], rtol=1e-10, atol=1e-15)
    assert np.array_equal(got["quant"], ref["quantiles"])
    assert np.allclose(got["mf"], ref["mean_field"], rtol=1e-13)
    assert np.allclose(got["var"], ref["var_field"], rtol=1e-12)
    assert np.array_equal(got["ex"], ref["exceedance"][0])
