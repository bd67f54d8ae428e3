"""GPU discrete adjoint against the oracle's FP64 adjoint (itself pinned by
finite differences in test_oracle_adjoint.py), on the same small problems:
gradients of a probe loss with respect to per-group omega_b and rigid
group ('site') positions.  Both adjoints get the same loss gradient dL/dp
(from the oracle's probe), so the comparison measures the reverse pass, not
the FP32 forward's effect on a small residual p - target.  Gradients are compared at
1e-4 relative to the largest component (FP32 forward and adjoint, FP64
reductions; the order of every cross-particle sum is fixed, so the
difference is FP32 rounding of a few hundred steps: measured on a GB300,
at most 5.3e-5 for the 1D site gradient, 1.8e-6 for the 1D omega_b
gradient, below 4e-7 in 2D).  The probe itself is compared at 1e-5.
Reruns give bit-identical gradients."""

GRAD_TOL = 1e-4
import numpy as np
import pytest

import oracle as O
from paper_2208_08038_gb300 import synth
from _common import gpu_from_workload
from test_oracle_adjoint import build_oracle, fd_problem, run_loss

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"


def oracle_gradients(D):
    wl, steps, groups = fd_problem(D)
    sp = wl.species[0]
    npts = len(wl.probe_nodes)
    om_true = synth.uniform_params(33, groups, 2.5, 3.5)
    _, target = run_loss(wl, steps, om_true, np.zeros((steps, npts)))
    s, sid, pid = build_oracle(wl, sp.omega_b)
    a = O.Adjoint(s, sid)
    L0, probe = a.forward(steps, pid, target)
    g_om, g_x = a.backward(groups, len(sp.x))
    a.close()
    s.close()
    g_site = np.stack([g_x[sp.pidx == k, :D].sum(axis=0) for k in range(groups)])
    return wl, steps, groups, target, probe, g_om, g_site


def gpu_problem(wl, steps, K):
    from paper_2208_08038_gb300.adjoint import SiteProblem
    sp = wl.species[0]
    ctx, sids, pid = gpu_from_workload(wl, deposit_mode=1, probe_cap=steps)
    prob = SiteProblem(ctx, sids[0], pid, sp.pidx, sp.x, sp.pidx, steps, K)
    return prob


@pytest.fixture(scope="module", params=[1, 2])
def case(request):
    return oracle_gradients(request.param)


def test_gpu_adjoint_matches_oracle(case):
    wl, steps, groups, target, probe_o, g_om, g_site = case
    D = wl.D
    prob = gpu_problem(wl, steps, K=20)
    sites0 = np.zeros((groups, D))
    probe = prob.run(wl.species[0].omega_b, sites0)
    assert np.abs(probe - probe_o).max() <= 1e-5 * np.abs(probe_o).max()
    go, gs = prob.gradients(2.0 * (probe_o - target), groups)
    assert np.abs(go - g_om).max() <= GRAD_TOL * np.abs(g_om).max(), (go, g_om)
    assert np.abs(gs - g_site).max() <= GRAD_TOL * np.abs(g_site).max(), (gs, g_site)


def test_checkpoint_interval_does_not_change_gradients(case):
    wl, steps, groups, target, probe_o, *_ = case
    out = []
    for K in (1, 7, steps):
        prob = gpu_problem(wl, steps, K=K)
        prob.run(wl.species[0].omega_b, np.zeros((groups, wl.D)))
        out.append(prob.gradients(2.0 * (probe_o - target), groups))
        prob.ctx.close()
    for go, gs in out[1:]:
        assert np.abs(go - out[0][0]).max() <= GRAD_TOL * np.abs(out[0][0]).max()
        assert np.abs(gs - out[0][1]).max() <= GRAD_TOL * np.abs(out[0][1]).max()


def test_gradients_bit_exact_rerun(case):
    """The adjoint's only cross-particle sums are the field-adjoint scatter
    and its per-cell accumulation (64-bit fixed point, integer adds) and the
    FP64 reductions (fixed order): two runs give identical gradients."""
    wl, steps, groups, target, probe_o, *_ = case
    out = []
    for _ in range(2):
        prob = gpu_problem(wl, steps, K=7)
        prob.run(wl.species[0].omega_b, np.zeros((groups, wl.D)))
        out.append(prob.gradients(2.0 * (probe_o - target), groups))
        prob.ctx.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_autograd_function(case):
    """The gradients through torch.autograd (PICProbe) of loss = sum_s,j
    w[s, j] probe[s, j], with w = 2 (p_oracle - target) fixed: the same
    dL/dprobe as test_gpu_adjoint_matches_oracle, so the oracle's gradients
    of that test apply, at the same tolerance; and bit-identical to the
    library's reverse pass called directly with that dL/dprobe."""
    import torch
    from paper_2208_08038_gb300.adjoint import PICProbe
    wl, steps, groups, target, probe_o, g_om, g_site = case
    sp = wl.species[0]
    w = 2.0 * (probe_o - target)
    prob = gpu_problem(wl, steps, K=16)
    om = torch.tensor(sp.omega_b, dtype=torch.float64, requires_grad=True)
    sites = torch.zeros((groups, wl.D), dtype=torch.float64, requires_grad=True)
    probe = PICProbe.apply(om, sites, prob)
    loss = (probe * torch.tensor(w, dtype=probe.dtype)).sum()
    loss.backward()
    assert np.abs(om.grad.numpy() - g_om).max() <= GRAD_TOL * np.abs(g_om).max()
    assert np.abs(sites.grad.numpy() - g_site).max() <= GRAD_TOL * np.abs(g_site).max()
    direct = gpu_problem(wl, steps, K=16)
    direct.run(sp.omega_b, np.zeros((groups, wl.D)))
    go, gs = direct.gradients(w.astype(np.float32), groups)
    assert np.array_equal(om.grad.numpy(), go)
    assert np.array_equal(sites.grad.numpy(), gs)
