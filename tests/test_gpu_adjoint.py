"""Second-order SW products and the adjoint of the switching work, on the GPU through the C ABI.

* Dual-number kernel: J w (J = dF/dx), (dF/dtheta) dtheta and the mixed product
  (d2U/dtheta dx) w against central differences of the FP64 oracle's forces (1e-7 relative).
* The adjoint context's own FP64 trajectory against the oracle's (Frenkel-Ladd and reversible
  scaling, NVT): W within 1e-9 relative, positions within 1e-8 A.
* dW/dtheta by the checkpointed adjoint against fourth-order central differences of the
  oracle's W(theta) over a short horizon (1e-6 relative, the chaos-free regime).
* Dot-product test over 2000 steps of a 32768-atom liquid at 1700 K: the adjoint gradient
  contracted with a random direction equals the tangent-linear derivative (1e-9 relative);
  this holds at any horizon because both are exact derivatives of the same discrete map.
* The checkpoint interval does not change the gradient (bit for bit).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_10449_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THETA0 = np.array(O.SW_SI[2:9], dtype=np.float64)
RCS = O.SW_SI[6] * O.SW_SI[1] + 0.5
CAP = 48


def _prm(theta):
    return (O.SW_SI[0], O.SW_SI[1], *theta, O.SW_SI[9])


def _sv(T):
    return math.sqrt(O.KB * T / (O.M_SI * O.MVV2E))


@pytest.fixture(scope="module")
def N():
    from paper_2103_10449_gb300 import nefe
    nefe.load()
    return nefe


def soa(a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a).T).reshape(-1), dtype=torch.float64, device="cuda")


def _dual(N, x, box, w, theta=THETA0, dtheta=None):
    n = len(x)
    xd, wd = soa(x), soa(w)
    nbr = torch.zeros(n * CAP, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    N.nefe_neighbor_build(xd, n, box, RCS, CAP, nbr, cnt)
    f = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    fd = torch.zeros_like(f)
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    N.nefe_sw_dual(xd, wd, n, box, RCS, nbr, cnt, CAP, N.params_from(_prm(theta)), dtheta, f, fd, out)
    torch.cuda.synchronize()
    return (f.cpu().numpy().reshape(3, n).T, fd.cpu().numpy().reshape(3, n).T, out.cpu().numpy())


def _oracle_F(x, box, theta=THETA0):
    return O.sw_energy(x, box, _prm(theta))[1]


@pytest.mark.parametrize("name", ["diamond216", "liquid512"])
def test_dual_products_match_oracle_differences(N, name):
    if name == "diamond216":
        x, box = I.diamond(3, 3, 3)
        x = I.rattle(x, 0.15, 31)
    else:
        x, box = I.liquid(512, 0.05425, seed=32)
    rng = np.random.default_rng(33)
    w = rng.standard_normal(x.shape)
    f, fd, out = _dual(N, x, box, w)
    e_o, f_o, _, _ = O.sw_energy(x, box, _prm(THETA0))
    assert abs(out[0] - e_o) <= 1e-10 * abs(e_o)
    assert np.abs(f - f_o).max() <= 1e-10 * np.abs(f_o).max()
    # E' = -F . w
    assert out[1] == pytest.approx(-np.sum(f_o * w), rel=1e-9)
    # J w against central differences of the oracle forces along w
    h = 1e-5
    jw = (8 * (_oracle_F(x + h * w, box) - _oracle_F(x - h * w, box))
          - (_oracle_F(x + 2 * h * w, box) - _oracle_F(x - 2 * h * w, box))) / (12 * h)
    assert np.abs(fd - jw).max() <= 1e-7 * np.abs(jw).max()
    # mixed product G'_m = sum_i w_i . d(dU/dx_i)/dtheta_m = -sum_i w_i . dF_i/dtheta_m
    for m in range(7):
        hm = 1e-5 * max(1.0, abs(THETA0[m]))
        tp, tm = THETA0.copy(), THETA0.copy()
        tp[m] += hm
        tm[m] -= hm
        dF = (_oracle_F(x, box, tp) - _oracle_F(x, box, tm)) / (2 * hm)
        ref = -np.sum(w * dF)
        assert abs(out[9 + m] - ref) <= 1e-6 * max(abs(ref), 1e-3 * np.abs(out[9:16]).max()), (m, out[9 + m], ref)


def test_dual_parameter_direction(N):
    """With w = 0: F' = (dF/dtheta) dtheta and E' = G . dtheta."""
    x, box = I.diamond(3, 3, 3)
    x = I.rattle(x, 0.1, 34)
    dth = np.array([0.3, -0.2, 0.1, 0.05, 0.01, 1.0, -0.05])
    f, fd, out = _dual(N, x, box, np.zeros_like(x), dtheta=dth)
    h = 1e-6
    ref = (_oracle_F(x, box, THETA0 + h * dth) - _oracle_F(x, box, THETA0 - h * dth)) / (2 * h)
    assert np.abs(fd - ref).max() <= 1e-6 * np.abs(ref).max()
    eref = (O.sw_energy(x, box, _prm(THETA0 + h * dth))[0] - O.sw_energy(x, box, _prm(THETA0 - h * dth))[0]) / (2 * h)
    assert out[1] == pytest.approx(eref, rel=1e-7)
    assert out[1] == pytest.approx(float(np.dot(out[2:9], dth)), rel=1e-12)


def _fl_setup(T=400.0):
    x0, box = I.diamond(2, 2, 2)
    v0 = I.gaussian_velocities(len(x0), _sv(T), 41)
    return x0, v0, box


def _oracle_run(x0, v0, box, theta, nst, kind, T=400.0, nsched=150):
    kw = dict(x=x0.copy(), v=v0.copy(), box=box.copy(), T=T, tdamp=0.1, seed=42, sys_id=3, prm=_prm(theta),
              nsched=nsched)
    if kind == "FL":
        s = O.System(sched=O.SCHED_FL, k_E=5.0, r0=x0.copy(), **kw)
    else:
        s = O.System(sched=O.SCHED_RS, lam_f=0.5, p_ext=1.0 / O.EV_A3_TO_GPA, **kw)
    return s.run(nst)


def _adjoint(N, x0, v0, box, kind, theta=THETA0, T=400.0, nsched=150, kc=45):
    common = dict(prm=N.params_from(_prm(theta)), T=T, tdamp=0.1, seed=42, sys_id=3, nsched=nsched,
                  checkpoint_every=kc)
    if kind == "FL":
        return N.Adjoint(x0, v0, box, kind=N.NEFE_SCHED_FL, r0=x0, k_E=5.0, **common)
    return N.Adjoint(x0, v0, box, kind=N.NEFE_SCHED_RS, lambda_f=0.5, P_GPa=1.0, **common)


@pytest.mark.parametrize("kind", ["FL", "RS"])
def test_adjoint_trajectory_matches_oracle(N, kind):
    x0, v0, box = _fl_setup()
    nst = 120
    orc = _oracle_run(x0, v0, box, THETA0, nst, kind)
    adj = _adjoint(N, x0, v0, box, kind)
    W = adj.forward(nst)
    x, v = adj.state()
    adj.close()
    assert W == pytest.approx(orc.W, rel=1e-9)
    assert np.abs(x - orc.x).max() < 1e-8
    assert np.abs(v - orc.v).max() < 1e-6


@pytest.mark.parametrize("kind", ["FL", "RS"])
def test_adjoint_gradient_matches_oracle_differences(N, kind):
    x0, v0, box = _fl_setup()
    nst = 100
    adj = _adjoint(N, x0, v0, box, kind, kc=16)
    adj.forward(nst)
    g = adj.backward()
    adj.close()
    g_fd = np.zeros(7)
    for m in range(7):
        h = 1e-5 * max(1.0, abs(THETA0[m]))

        def W(d):
            t = THETA0.copy()
            t[m] += d
            return _oracle_run(x0, v0, box, t, nst, kind).W
        g_fd[m] = (8 * (W(h) - W(-h)) - (W(2 * h) - W(-2 * h))) / (12 * h)
    assert np.abs(g - g_fd).max() <= 1e-6 * np.abs(g_fd).max(), (g, g_fd)


def test_checkpoint_interval_leaves_gradient_bitwise(N):
    x0, v0, box = _fl_setup()
    nst = 90
    grads = []
    for kc in (1, 7, 45, 90):
        adj = _adjoint(N, x0, v0, box, "FL", kc=kc)
        adj.forward(nst)
        grads.append(adj.backward(initial_state=True))
        adj.close()
    for g in grads[1:]:
        for a, b in zip(g, grads[0]):
            assert np.array_equal(a, b)


def test_switching_work_autograd(N):
    from paper_2103_10449_gb300.autograd import switching_work
    x0, v0, box = _fl_setup()
    adj = _adjoint(N, x0, v0, box, "FL")
    th = torch.tensor(THETA0, dtype=torch.float64, requires_grad=True)
    W = switching_work(th, adj, 60)
    W.backward()
    adj2 = _adjoint(N, x0, v0, box, "FL")
    W2 = adj2.forward(60)
    g2 = adj2.backward()
    adj.close()
    adj2.close()
    assert W.item() == W2
    assert np.array_equal(th.grad.numpy(), g2)


def test_dot_product_liquid_32768_1700K_2000_steps(N):
    """Adjoint against tangent-linear over the full differentiation workload (liquid Si,
    32768 atoms, 1700 K, reversible scaling 1 -> 0.5 over 2000 steps, checkpoints every 45)."""
    x, box = I.liquid(32768, 0.05425, seed=51)
    v = I.gaussian_velocities(len(x), _sv(1700.0), 52)
    ctx = N.Context(precision=N.NEFE_FP32)
    s = ctx.add_system(x, box, v=v)
    ctx.set_thermostat(s, 1700.0, 0.1, 53)
    ctx.run(1500)
    x0, v0, _ = ctx.get_state(s)
    ctx.close()
    adj = N.Adjoint(x0, v0, box, kind=N.NEFE_SCHED_RS, lambda_f=0.5, T=1700.0, tdamp=0.1, seed=54, nsched=2000,
                    checkpoint_every=45)
    K = 2000
    W = adj.forward(K)
    g, gx, gv = adj.backward(initial_state=True)
    rng = np.random.default_rng(55)
    dth = rng.standard_normal(7) * np.maximum(np.abs(THETA0), 0.1) * 1e-3
    dx0 = rng.standard_normal(x0.shape) * 1e-3
    dv0 = rng.standard_normal(v0.shape) * 1e-1
    W2, dW = adj.tangent(K, dth, dx0, dv0)
    adj.close()
    assert W2 == W
    terms = np.array([np.dot(g, dth), np.sum(gx * dx0), np.sum(gv * dv0)])
    assert np.isfinite(terms).all() and np.isfinite(dW)
    assert abs(terms.sum() - dW) <= 1e-9 * np.abs(terms).sum(), (terms, dW)
