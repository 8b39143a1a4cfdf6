"""The coupler optimisation pipeline (Sec. 4, Fig. 4 analogue) end to end on
a small grid: the differentiable transmission against central differences of
itself, and a few NAdam iterations that raise it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2603_24027_gb300 import build as B
    B.build()
    from paper_2603_24027_gb300 import design
    return design


def small_problem(D, tape=("f32", 1, "linear")):
    from paper_2603_24027_gb300 import _capi as A
    from paper_2603_24027_gb300 import inputs as I
    w = I.coupler(nx=60, ny=44, nz=36, P=6, n_steps=260, dx=20e-9, dev=24, wg_w=8, layer=5,
                  src_dz=7, det_dz=4)
    return D.Coupler(w, A.record_cfg(*tape), sigma_cells=1.5)


def test_transmission_gradient_against_central_differences(D):
    prob = small_problem(D)
    rng = np.random.default_rng(1)
    theta0 = rng.uniform(0.2, 0.8, prob.shape2d)
    theta = torch.tensor(theta0, dtype=torch.float64, device="cuda", requires_grad=True)
    T = prob.transmission(theta, 1.0)
    T.backward()
    g = theta.grad.cpu().numpy()
    assert float(T.detach()) > 0 and np.isfinite(g).all()
    # along the gradient direction the derivative is |g|, far above FP32 noise
    d = g / np.linalg.norm(g)
    h = 0.05
    with torch.no_grad():
        tp = float(prob.transmission(torch.tensor(theta0 + h * d, device="cuda"), 1.0))
        tm = float(prob.transmission(torch.tensor(theta0 - h * d, device="cuda"), 1.0))
    fd = (tp - tm) / (2 * h)
    assert fd == pytest.approx(np.linalg.norm(g), rel=2e-2)


def test_a_few_iterations_raise_the_transmission(D):
    prob = small_problem(D, ("e4m3b11fnuz", 4, "linear"))
    theta0 = np.random.default_rng(0).uniform(0.0, 1.0, prob.shape2d)
    _, hist, final = D.optimise(prob, theta0, iters=8, lr=0.05, warmup=2, beta_switch=100)
    assert hist[-1] > hist[0] + 0.1, hist
