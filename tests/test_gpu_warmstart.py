"""What the learned warm start gains: a small U-Net trained on steady
cavities from the batched solver cuts the steps to the same residual on
held-out cavities, and the solver still lands on the same steady state."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08591_gb300 import _build
    _build.build()


def test_warm_start_reduces_steps_to_steady():
    from paper_2108_08591_gb300 import warmstart
    r = warmstart.study(side=32, n_train=32, n_test=8, U=0.1, re_range=(20.0, 200.0), tol=1e-7,
                        max_steps=400_000, check_every=50, epochs=120, channels=(16, 32, 64),
                        batch=8, lr=2e-3, seed=5)
    print(r)
    assert r["n_train_converged"] == 32 and r["n_test_converged_both"] == 8
    assert r["warm_steps_mean"] < 0.7 * r["cold_steps_mean"], r
    assert r["final_warm_vs_cold_u_max"] < 1e-4, r
    assert r["pred_err_u_mean"] < 0.2, r
    assert r["n_test_converged_neq"] == 8 and r["warm_neq_steps_mean"] < 0.7 * r["cold_steps_mean"], r
