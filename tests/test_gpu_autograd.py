"""Differentiation of the SW energy on the GPU: forces and dE/d(A, B, p, q, a, lambda3, gamma)
against the FP64 oracle (forces element by element; parameter derivatives against fourth-order
central differences of the oracle's energy, whose truncation and rounding errors at the steps
used are below 1e-9 relative)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_10449_gb300 import inputs as I

torch = pytest.importorskip("torch")

THETA0 = np.array(O.SW_SI[2:9], dtype=np.float64)       # A, B, p, q, a, lambda3, gamma
FIXED = (O.SW_SI[0], O.SW_SI[1], O.SW_SI[9])


def _prm(theta):
    return (FIXED[0], FIXED[1], *theta, FIXED[2])


def _fd_grad(x, box, theta):
    g = np.zeros(7)
    for k in range(7):
        h = 1e-5 * max(1.0, abs(theta[k]))

        def e(d):
            t = theta.copy()
            t[k] += d
            return O.sw_energy(x, box, _prm(t))[0]
        g[k] = (8.0 * (e(h) - e(-h)) - (e(2 * h) - e(-2 * h))) / (12.0 * h)
    return g


def _cases():
    x, b = I.diamond(3, 3, 3)
    yield "diamond216", I.rattle(x, 0.15, 21), b, THETA0
    x, b = I.liquid(512, 0.05425, seed=22)
    t = THETA0.copy()
    t[3] = 0.5            # a non-zero attractive exponent exercises dE/dq's s^-q ln s term
    yield "liquid512_q05", x, b, t


CASES = {name: (x, b, t) for name, x, b, t in _cases()}


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(CASES))
def test_energy_forces_and_parameter_gradient_fp64(name):
    from paper_2103_10449_gb300.autograd import sw_energy
    x, box, theta = CASES[name]
    xd = torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device="cuda", requires_grad=True)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    E = sw_energy(xd, th, box, fixed=FIXED)
    E.backward()
    e_o, f_o, _, _ = O.sw_energy(x, box, _prm(theta))
    assert abs(E.item() - e_o) <= 1e-10 * abs(e_o)
    f = -xd.grad.cpu().numpy().T
    assert np.abs(f - f_o).max() <= 1e-10 * np.abs(f_o).max()
    g_fd = _fd_grad(x, box, theta)
    g = th.grad.numpy()
    scale = np.abs(g_fd).max()
    assert np.abs(g - g_fd).max() <= 1e-8 * scale, (g, g_fd)


@pytest.mark.gpu
def test_parameter_gradient_fp32_close():
    from paper_2103_10449_gb300 import nefe as N
    from paper_2103_10449_gb300.autograd import sw_energy
    x, box, theta = CASES["diamond216"]
    xd = torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device="cuda")
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    E = sw_energy(xd, th, box, fixed=FIXED, precision=N.NEFE_FP32)
    (g,) = torch.autograd.grad(E, th)
    g_fd = _fd_grad(x, box, theta)
    assert np.abs(g.numpy() - g_fd).max() <= 2e-5 * np.abs(g_fd).max()


@pytest.mark.gpu
def test_gradient_chains_through_a_loss():
    """d(c E^2)/dx = 2 c E dE/dx: the backward scales by the incoming gradient."""
    from paper_2103_10449_gb300.autograd import sw_energy
    x, box, theta = CASES["diamond216"]
    xd = torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device="cuda", requires_grad=True)
    th = torch.tensor(theta, dtype=torch.float64)
    E = sw_energy(xd, th, box, fixed=FIXED)
    (gx1,) = torch.autograd.grad(E, xd, retain_graph=True)
    (gx2,) = torch.autograd.grad(0.25 * E * E, xd)
    assert torch.allclose(gx2, 0.5 * E.detach() * gx1, rtol=1e-14, atol=0)


def test_cpu_tensor_is_rejected():
    """No CPU fallback: positions must live on the device."""
    from paper_2103_10449_gb300.autograd import sw_energy
    x, box = I.diamond(2, 2, 2)
    with pytest.raises(ValueError):
        sw_energy(torch.tensor(x.T.copy()), None, box)
