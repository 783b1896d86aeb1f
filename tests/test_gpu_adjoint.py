"""The hand-written adjoint (through the C ABI and the torch.autograd.Function)
against the FP64 oracle's complex-step gradient and against central finite
differences, and the calibration of r_b and a it enables.

J = mean_x sum_y u_x after N steps of a periodic body-force channel;
gradients with respect to r_b, the Bosanquet factor a and the body force G.
* FP64 adjoint vs oracle complex step (exact to round-off): 1e-9 relative;
* FP32 adjoint (FP32 states, FP64 parameter sums) vs oracle: 1e-4 relative;
* the 64-row channel of Sec. 3.1 at Kn 0.1, 0.5, 1.0, 20000 steps with a
  checkpoint every 141 steps: adjoint vs central differences of FP64 forward
  runs with h = 1e-4 relative, within 1e-4 (G is tested on J, which is linear
  in G to first order, not on Q = J/(3 G ny^2 sqrt(1/6)), whose G-derivative
  nearly vanishes);
* Gauss-Newton on the adjoint gradients recovers r_b and a from a Q(Kn)
  curve that the oracle computed with seed-chosen true values.
"""
import math

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_01955_gb300.clb as clb

    return clb


def gpu_grad(clb, nx, ny, kn, a, r, g, n, storage, every=0):
    fg = clb.FlowGradient(nx, ny, kn, a, r, g, n, storage=storage, checkpoint_every=every)
    J = fg.J
    grad = fg.grad()
    again = fg.grad()  # a second backward pass gives the same numbers
    fg.close()
    assert grad == again  # fixed summation order: the same bits
    return J, dict(zip(("r", "a", "g"), grad))


CASES = [(4, 8, 0.1, 0.7, 1e-5), (1, 5, 0.5, 0.5, -2e-5), (3, 8, 1.0, 0.95, 3e-5)]


@pytest.mark.parametrize("nx,ny,kn,r,G", CASES)
def test_fp64_adjoint_matches_oracle_complex_step(clb, oracle_mod, nx, ny, kn, r, G):
    n = 1500
    J, g = gpu_grad(clb, nx, ny, kn, 2.0, r, G, n, "fp64", every=37)
    Jo, go = oracle_mod.gradient_cs(oracle_mod.OracleParams(nx=nx, ny=ny, kn=kn, r=r, gx=G), n)
    assert J == pytest.approx(Jo, rel=1e-12)
    for k in ("r", "a", "g"):
        assert g[k] == pytest.approx(go[k], rel=1e-9), k


@pytest.mark.parametrize("nx,ny,kn,r,G", CASES)
def test_fp32_adjoint_matches_oracle(clb, oracle_mod, nx, ny, kn, r, G):
    n = 1500
    J, g = gpu_grad(clb, nx, ny, kn, 2.0, r, G, n, "fp32s")
    Jo, go = oracle_mod.gradient_cs(oracle_mod.OracleParams(nx=nx, ny=ny, kn=kn, r=r, gx=G), n)
    assert J == pytest.approx(Jo, rel=1e-5)
    for k in ("r", "a", "g"):
        assert g[k] == pytest.approx(go[k], rel=1e-4), k


@pytest.mark.parametrize("kn", [0.1, 0.5, 1.0])
def test_adjoint_vs_central_differences_64_rows(clb, kn):
    nx, ny, n, a, G = 4, 64, 20000, 2.0, 1e-6
    r = 0.628092213  # Eq. 21 at sigma = 1 (B1 = 0.8183)
    J, g32 = gpu_grad(clb, nx, ny, kn, a, r, G, n, "fp32s", every=141)

    def J64(**kw):
        p = dict(a=a, r=r, g=G)
        p.update(kw)
        fg = clb.FlowGradient(nx, ny, kn, p["a"], p["r"], p["g"], n, storage="fp64", checkpoint_every=141)
        v = fg.J
        fg.close()
        return v

    base = dict(r=r, a=a, g=G)
    for k in ("r", "a", "g"):
        h = 1e-4 * abs(base[k])
        fd = (J64(**{k: base[k] + h}) - J64(**{k: base[k] - h})) / (2 * h)
        assert g32[k] == pytest.approx(fd, rel=1e-4), (k, g32[k], fd)


def test_flow_rate_autograd(clb):
    import torch

    cfg = dict(nx=4, ny=16, kn=0.5, nsteps=3000, storage="fp64")
    r = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
    a = torch.tensor(2.0, dtype=torch.float64, requires_grad=True)
    g = torch.tensor(2e-6, dtype=torch.float64, requires_grad=True)
    q = clb.flow_rate(r, a, g, cfg)
    q.backward()
    norm = 3 * 2e-6 * 16**2 * math.sqrt(1 / 6)
    fg = clb.FlowGradient(4, 16, 0.5, 2.0, 0.7, 2e-6, 3000, storage="fp64")
    dr, da, dg = fg.grad()
    assert q.item() == pytest.approx(fg.J / norm, rel=1e-14)
    assert float(r.grad) == pytest.approx(dr / norm, rel=1e-12)
    assert float(a.grad) == pytest.approx(da / norm, rel=1e-12)
    assert float(g.grad) == pytest.approx(dg / norm - q.item() / 2e-6, rel=1e-6, abs=1e-6 * abs(q.item()) / 2e-6)
    fg.close()


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-12), ("fp32s", 1e-5)])
@pytest.mark.parametrize("nx,ny,n,every", [(4, 16, 700, 31), (3, 5, 1000, 0), (4, 64, 2000, 45)])
def test_resident_engine_matches_per_step_launches(clb, storage, tol, nx, ny, n, every):
    """The one-block-per-pass engine (grids that fit in shared memory) and the
    one-launch-per-step engine compute the same states; only the order of the
    FP64 sums of J and of the gradient differs."""
    out = []
    for pipeline in (0, 1):
        fg = clb.FlowGradient(nx, ny, 0.3, 2.0, 0.8, 2e-5, n, storage=storage, checkpoint_every=every,
                              pipeline=pipeline)
        out.append((fg.J, fg.grad()))
        fg.close()
    (j0, g0), (j1, g1) = out
    assert j0 == pytest.approx(j1, rel=tol)
    for a, b in zip(g0, g1):
        assert a == pytest.approx(b, rel=tol)


def test_q_and_its_gradient_match_oracle(clb, oracle_mod):
    """Q (clb_adjoint_q) against the oracle's own Q observable, and dQ/d(r_b,
    a, G) (clb_adjoint_q_backward) against the oracle's complex-step dJ
    divided by the same normalisation (for G, minus Q/G); two backward calls
    give the same bits."""
    nx, ny, kn, r, G, n = 3, 8, 0.5, 0.8, 2e-5, 1500
    fg = clb.FlowGradient(nx, ny, kn, 2.0, r, G, n, storage="fp64", checkpoint_every=37)
    q = fg.q_norm
    dq = fg.q_grad()
    again = fg.q_grad(2.0)
    fg.close()
    assert again == [2.0 * v for v in dq]
    s = oracle_mod.OracleSim(oracle_mod.OracleParams(nx=nx, ny=ny, kn=kn, r=r, gx=G))
    s.step(n, 1)
    qo = s.observables()["q_norm"]
    assert q == pytest.approx(qo, rel=1e-12)
    Jo, go = oracle_mod.gradient_cs(oracle_mod.OracleParams(nx=nx, ny=ny, kn=kn, r=r, gx=G), n)
    norm = Jo / qo
    assert dq[0] == pytest.approx(go["r"] / norm, rel=1e-9)
    assert dq[1] == pytest.approx(go["a"] / norm, rel=1e-9)
    assert dq[2] == pytest.approx(go["g"] / norm - qo / G, rel=1e-6, abs=1e-9 * qo / abs(G))


def test_calibration_recovers_r_and_a(clb, oracle_mod):
    """Fit (r_b, a) to Q at Kn = 0.1, 0.5, 1.0 (ny = 64, 20000 steps) generated
    by the oracle from seed-chosen true values, by Gauss-Newton on the FP32
    adjoint gradients."""
    r_rng = inputs.rng(7)
    r_true = float(r_rng.uniform(0.5, 0.9))
    a_true = float(r_rng.uniform(1.5, 2.5))
    kns, ny, n, G = (0.1, 0.5, 1.0), 64, 20000, 1e-6
    target = []
    for kn in kns:
        s = oracle_mod.OracleSim(oracle_mod.OracleParams(nx=1, ny=ny, kn=kn, r=r_true, a=a_true, gx=G))
        s.step(n, 1)
        target.append(s.observables()["q_norm"])
    target = np.array(target)
    theta = np.array([0.6, 1.0])  # start: r_b, a
    loss0 = None
    for it in range(12):
        res, jac = [], []
        for kn, qt in zip(kns, target):
            fg = clb.FlowGradient(4, ny, kn, theta[1], theta[0], G, n, storage="fp32s", checkpoint_every=141)
            q = fg.q_norm
            dr, da, _ = fg.q_grad()
            fg.close()
            res.append(q / qt - 1)
            jac.append([dr / qt, da / qt])
        res, jac = np.array(res), np.array(jac)
        loss = float(res @ res)
        loss0 = loss if loss0 is None else loss0
        step, *_ = np.linalg.lstsq(jac, -res, rcond=None)
        theta = theta + step
        theta[0] = min(max(theta[0], 0.05), 1.0)
        if np.abs(step).max() < 1e-7:
            break
    assert loss < 1e-8 * loss0 or loss < 1e-14
    assert theta[0] == pytest.approx(r_true, abs=1e-3)
    assert theta[1] == pytest.approx(a_true, abs=1e-2)
