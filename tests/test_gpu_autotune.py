"""The autotuner times candidate multigrid schedules on a short solve (then,
for the winner, operator reuse factors, residual tile heights and the
temporally blocked legs) and returns the fastest one that converged."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_tune_level_returns_a_converging_schedule(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_17018_gb300 import autotune as A
    best, table = A.tune_level(0, 64, "fp32mg", steps=2, reps=1, splits=(1, 2))
    n = len(A.CANDIDATES["vcycles"]) * len(A.CANDIDATES["nu"]) * len(A.CANDIDATES["small_cells"])
    assert len(table) == n * 2 + len(A.CANDIDATES["jac_lag"]) + len(A.CANDIDATES["keep_lags"]) - 1 + len(
        [r for r in A.CANDIDATES["res_rows"] if r]) + len([t for t in A.CANDIDATES["tb_cells"] if t])
    lag0 = max(A.CANDIDATES["keep_lags"])
    assert all(r["jac_lag"] == lag0 and r["jac_keep"] == 1 for r in table[:n * 2])
    assert {r["mg_small_cells"] for r in table} == set(A.CANDIDATES["small_cells"])
    assert best["failed"] == 0 and best["solves_per_s"] > 0
    assert best["solves_per_s"] == max(r["solves_per_s"] for r in table if r["failed"] == 0)
    path = str(tmp_path / "cache.json")
    A.save_cache({"k": best}, path)
    assert A.load_cache(path) == {"k": best}
