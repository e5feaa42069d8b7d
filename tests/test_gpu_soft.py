"""Soft-deposit mode on the GPU: deposits against the oracle, the adjoint
kernel's gradient against the oracle's FP64 reverse sweep and against central
finite differences (h = 1e-3 in log-parameters), and the autograd.Function."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2506_23364_gb300 as awo
from paper_2506_23364_gb300 import inputs

pytestmark = pytest.mark.gpu

MU0, K0 = math.tan(math.radians(25.0)), 1e-3


@pytest.fixture(scope="module")
def problem():
    z = inputs.fbm(112, 0.8, seed=21, relief=900.0, m=97).astype(np.float32)
    prob = awo.SoftOverlay(z, 10.0, (30.0, 50.0), traj_per_cell=16, max_steps=400, persistence=0.85,
                           randomness=0.2, seed=5)
    cells = prob.cells[: prob.n_cells].cpu().numpy().view(np.uint32)
    w = np.random.default_rng(3).uniform(0.5, 1.5, cells.size).astype(np.float32)
    op = lambda mu, k: oracle.SimParams(mu=mu, drag_k=k, persistence=0.85, randomness=0.2, traj_per_cell=16,
                                        max_steps=400, seed=5)
    return z, prob, cells, w, op


def test_soft_forward_matches_oracle_and_conserves_mass(problem):
    z, prob, cells, w, op = problem
    assert cells.size > 200
    wt = torch.from_numpy(w).cuda()
    D = prob.forward_raw(MU0, K0, wt).cpu().numpy()
    q = prob.q.cpu().numpy()
    Wq = np.rint(w.astype(np.float64) * 2.0 ** 32).astype(np.int64)
    assert int(q.sum()) == 16 * int(Wq.sum())  # every particle deposits exactly round(w 2^32)
    Dref, st = oracle.soft_forward(z, 10.0, cells, w.astype(np.float64), op(MU0, K0), threads=8)
    assert np.allclose(D, Dref, rtol=1e-4, atol=2e-5)
    assert prob.stats.cpu().tolist()[1] == st["n_traj"]
    D2 = prob.forward_raw(MU0, K0, wt).cpu().numpy()
    assert np.array_equal(D, D2)


# Error model of the adjoint against the oracle's FP64 reverse sweep.  The
# kernel keeps each particle's energy, survival and tangents in FP32 and
# reduces over particles in FP64.  Every move applies a fixed number of FP32
# roundings (unit u = 2^-24) to that state, so a particle's term carries a
# relative error of at most c n u after n moves; the FP64 sums add nothing
# measurable.  A gradient component is therefore off by at most
# c u n_mean A, with A the oracle's sum over particles of |term| (the
# conditioning of the sum: relative errors are c u n_mean A / |sum|).
# Measured on GB300: c <= 9 over the cases below; the tests allow c = 32.
# A weight's gradient is a sum over that entry's particles of terms bounded
# by max|G|, hence off by at most c u n_mean of the largest weight gradient.
C_FP32 = 32.0
U32 = 2.0 ** -24


def _check_adjoint(prob, gt, gw, rt, rw, ra):
    st = prob.stats.cpu().tolist()
    n_mean = st[0] / st[1]
    bound = C_FP32 * U32 * n_mean * ra
    assert np.all(np.abs(gt - rt) <= bound), (gt, rt, bound)
    assert np.max(np.abs(gw - rw)) <= C_FP32 * U32 * n_mean * np.abs(rw).max()


@pytest.mark.parametrize("gseed", [9, 10, 11])
def test_adjoint_matches_fp64_reverse_sweep(problem, gseed):
    z, prob, cells, w, op = problem
    wt = torch.from_numpy(w).cuda()
    G = np.random.default_rng(gseed).normal(size=z.shape).astype(np.float32)
    gt, gw = prob.backward_raw(MU0, K0, wt, torch.from_numpy(G).cuda())
    gt, gw = gt.cpu().numpy(), gw.cpu().numpy()
    rt, rw, ra = oracle.soft_gradient(z, 10.0, cells, w.astype(np.float64), op(MU0, K0), G.astype(np.float64),
                                      threads=8, with_abs=True)
    _check_adjoint(prob, gt, gw, rt, rw, ra)


def test_adjoint_matches_central_differences(problem):
    z, prob, cells, w, op = problem
    wt = torch.from_numpy(w).cuda()
    Dstar = prob.forward_raw(MU0 * 1.2, K0 * 0.8, wt)
    L = lambda mu, k: float(((prob.forward_raw(mu, k, wt) - Dstar) ** 2).sum())
    D0 = prob.forward_raw(MU0, K0, wt)
    gt, _ = prob.backward_raw(MU0, K0, wt, 2.0 * (D0 - Dstar))
    gt = gt.cpu().numpy()
    h = 1e-3
    fd_mu = (L(MU0 * math.exp(h), K0) - L(MU0 * math.exp(-h), K0)) / (2 * h)
    fd_k = (L(MU0, K0 * math.exp(h)) - L(MU0, K0 * math.exp(-h))) / (2 * h)
    assert abs(gt[0] - fd_mu) <= 5e-3 * abs(fd_mu), (gt[0], fd_mu)
    assert abs(gt[1] - fd_k) <= 5e-3 * abs(fd_k), (gt[1], fd_k)


def test_autograd_function(problem):
    z, prob, cells, w, op = problem
    wt = torch.from_numpy(w).cuda()
    Dstar = prob.forward_raw(MU0 * 1.2, K0 * 0.8, wt)
    log_mu = torch.tensor(math.log(MU0), dtype=torch.float64, requires_grad=True)
    log_k = torch.tensor(math.log(K0), dtype=torch.float64, requires_grad=True)
    wr = wt.clone().requires_grad_(True)
    D = prob.deposit(log_mu, log_k, wr)
    loss = ((D - Dstar) ** 2).sum()
    loss.backward()
    gt, gw = prob.backward_raw(MU0, K0, wt, 2.0 * (D.detach() - Dstar))
    assert torch.allclose(torch.stack([log_mu.grad, log_k.grad]), gt.cpu(), rtol=1e-12, atol=0)
    assert torch.equal(wr.grad, gw)


# ----------------------------------------------------------------------------
# The differentiable workload's own shape: 1024^2 fBm DEM (uint16 dm), release
# range of the 2048^2 workload, 128 particles per release cell, cap 2048,
# release weights U(0.5, 1.5), target at hidden parameters (1.2 mu0, 0.8 k0).
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def problem1024():
    n = 1024
    dem = inputs.quantise_dm(inputs.fbm(n, 0.8, seed=3, relief=3000.0 * (n / 2048.0) ** 0.8))
    prob = awo.SoftOverlay(dem, 10.0, inputs.MID_RELEASE_DEG, traj_per_cell=128, max_steps=2048, seed=0)
    cells = prob.cells[: prob.n_cells].cpu().numpy().view(np.uint32)
    w = np.random.default_rng(3).uniform(0.5, 1.5, cells.size).astype(np.float32)
    op = lambda mu, k: oracle.SimParams(mu=mu, drag_k=k, traj_per_cell=128, max_steps=2048, seed=0)
    return oracle.decode_u16(dem), prob, cells, w, op


def test_differentiable_config_forward_against_oracle(problem1024):
    h, prob, cells, w, op = problem1024
    wt = torch.from_numpy(w).cuda()
    D = prob.forward_raw(MU0, K0, wt).cpu().numpy()
    Dref, st = oracle.soft_forward(h, 10.0, cells, w.astype(np.float64), op(MU0, K0), threads=16)
    steps, n_traj = prob.stats.cpu().tolist()[:2]
    assert n_traj == st["n_traj"]
    # a particle ends once its survival falls below 1e-7: FP32 survival on the
    # GPU and FP64 in the oracle may cross that threshold one move apart
    assert abs(steps - st["total_steps"]) <= 1e-5 * st["total_steps"]
    assert st["n_traj"] == 128 * cells.size > 5_000_000
    assert np.abs(D - Dref).max() <= 1e-5 * np.abs(Dref).max()
    q = prob.q.cpu().numpy()
    assert int(q.sum()) == 128 * int(np.rint(w.astype(np.float64) * 2.0 ** 32).astype(np.int64).sum())


@pytest.mark.parametrize("which", ["random", "fit"])
def test_differentiable_config_adjoint_against_fp64_sweep(problem1024, which):
    """The 1024^2, 128-particle configuration: the adjoint against the FP64
    reverse sweep, for a random G and for the fit's own G = 2 (D - D*)."""
    h, prob, cells, w, op = problem1024
    wt = torch.from_numpy(w).cuda()
    if which == "random":
        G = torch.from_numpy(np.random.default_rng(3).normal(size=h.shape).astype(np.float32)).cuda()
    else:
        Dstar = prob.forward_raw(MU0 * 1.2, K0 * 0.8, wt)
        G = (2.0 * (prob.forward_raw(MU0, K0, wt) - Dstar)).to(torch.float32)
    gt, gw = prob.backward_raw(MU0, K0, wt, G)
    gt, gw = gt.cpu().numpy(), gw.cpu().numpy()
    rt, rw, ra = oracle.soft_gradient(h, 10.0, cells, w.astype(np.float64), op(MU0, K0),
                                      G.cpu().numpy().astype(np.float64), threads=16, with_abs=True)
    _check_adjoint(prob, gt, gw, rt, rw, ra)
    if which == "fit":  # a well-conditioned sum (A / |sum| < 10): close in relative terms too
        assert np.all(np.abs(gt - rt) <= 1e-4 * np.abs(rt)), (gt, rt)


def test_differentiable_config_central_differences(problem1024):
    """Central differences in log-parameters (h = 1e-3) of the fit's loss."""
    h_, prob, cells, w, op = problem1024
    wt = torch.from_numpy(w).cuda()
    Dstar = prob.forward_raw(MU0 * 1.2, K0 * 0.8, wt)
    L = lambda mu, k: float(((prob.forward_raw(mu, k, wt) - Dstar) ** 2).sum())
    gt, _ = prob.backward_raw(MU0, K0, wt, 2.0 * (prob.forward_raw(MU0, K0, wt) - Dstar))
    gt = gt.cpu().numpy()
    h = 1e-3
    fd = [(L(MU0 * math.exp(h), K0) - L(MU0 * math.exp(-h), K0)) / (2 * h),
          (L(MU0, K0 * math.exp(h)) - L(MU0, K0 * math.exp(-h))) / (2 * h)]
    for i in range(2):
        assert abs(gt[i] - fd[i]) <= 1e-3 * abs(fd[i]), (i, gt[i], fd[i])
