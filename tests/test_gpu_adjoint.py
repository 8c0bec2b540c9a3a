"""Force adjoint (force-matching gradients) vs the oracle, through the C ABI.

The oracle differentiates its FP64 forces by the complex-step method (exact
to rounding, pinned by finite differences in test_oracle_pins); the CUDA
adjoint forms the Hessian-vector product and the (lambda, epsilon, sigma)
derivatives analytically in FP32 from recomputed leg and triplet terms.
Tolerance (derived from the arithmetic): second derivatives carry the FP32
cancellation of the forces once more, so dL/dx is held to 1e-4 per atom
relative to max(|ref_i|, rms(ref)) and dL/dtheta to 1e-4 relative (dL/depsilon
against the magnitude of its two cancelling parts, see _check_theta).
"""
import math

import numpy as np
import pytest

from paper_0809_2811_gb300 import inputs as I

pytestmark = pytest.mark.gpu

G_TOL = 1e-4


def _rel_err_rows(g, r):
    mag = np.linalg.norm(r, axis=1)
    den = np.maximum(mag, math.sqrt(np.mean(mag ** 2)))
    return float((np.linalg.norm(g - r, axis=1) / den).max())


def _check_theta(orc, x, box, w, gt, gt_ref, prm=None):
    """dL/dlambda and dL/dsigma relative; dL/depsilon = -(D2 + D3)/epsilon is a
    cancelling sum like E2 + E3, so it is judged against (|D2| + |D3|)/epsilon
    (D2 from the oracle at lambda = 0, D3 = -lambda dL/dlambda)."""
    p = orc.default_params() if prm is None else prm
    p0 = p.copy()
    p0[0] = 0.0
    _, g2 = orc.force_vjp(x, box, w, p0)
    d2 = -p[1] * g2[1]
    d3 = -p[0] * gt_ref[0]
    assert abs(gt[0] - gt_ref[0]) <= G_TOL * abs(gt_ref[0])
    assert abs(gt[1] - gt_ref[1]) <= G_TOL * (abs(d2) + abs(d3)) / p[1]
    assert abs(gt[2] - gt_ref[2]) <= G_TOL * abs(gt_ref[2])


def _gpu_vjp(mwlib, torch, n, box, x, w, prm=None):
    s = mwlib.System(n, box)
    try:
        if prm is not None:
            s.set_params(prm)
        s.set_state(x)
        s.energy_forces()
        wd = torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda()
        gx = torch.empty_like(wd)
        torch.cuda.synchronize()
        gt = mwlib.mw_energy_forces_vjp(s.h, wd, gx, s.nbox)
        torch.cuda.synchronize()
        return gx.cpu().numpy().astype(np.float64), gt
    finally:
        s.close()


CASES = {
    "liquidlike_1000": lambda: I.jittered_box(1000, 1.0, 0.25, 501),
    "dense_729": lambda: I.jittered_box(729, 1.10, 0.25, 502),
    "ice_ih_288_jitter": lambda: (lambda xb: (xb[0] + np.random.default_rng(3).normal(0, 0.05, xb[0].shape), xb[1]))(
        I.ice_ih(4, 3, 3, 0.92)),
    "ragged_1237": lambda: I.jittered_box(1237, 0.97, 0.2, 503),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_adjoint_matches_oracle(mwlib, orc, case):
    torch = pytest.importorskip("torch")
    x, box = CASES[case]()
    x = I.snap_to_grid(x, box)
    w = np.random.default_rng(11).normal(size=x.shape)
    gx_ref, gt_ref = orc.force_vjp(x, box, w)
    gx, gt = _gpu_vjp(mwlib, torch, len(x), box, x, w)
    assert _rel_err_rows(gx, gx_ref) <= G_TOL
    _check_theta(orc, x, box, w, gt[0], gt_ref)


def test_adjoint_dense_overflow_path(mwlib, orc):
    """More than 24 legs per centre: the overflow adjoint kernel takes those centres."""
    torch = pytest.importorskip("torch")
    x, box = I.jittered_box(512, 3.5, 0.1, 104)
    x = I.snap_to_grid(x, box)
    w = np.random.default_rng(12).normal(size=x.shape)
    gx_ref, gt_ref = orc.force_vjp(x, box, w)
    gx, gt = _gpu_vjp(mwlib, torch, len(x), box, x, w)
    assert _rel_err_rows(gx, gx_ref) <= G_TOL
    _check_theta(orc, x, box, w, gt[0], gt_ref)


def test_adjoint_at_perturbed_parameters_batch(mwlib, orc):
    """Force-matching start point lambda = 21, epsilon and sigma x 1.05, on a batch."""
    torch = pytest.importorskip("torch")
    n = [343, 400, 512]
    xs, boxes = [], []
    for k, nn in enumerate(n):
        x, b = I.jittered_box(nn, 0.9998, 0.2, 600 + k)
        xs.append(I.snap_to_grid(x, b))
        boxes.append(b)
    w = np.random.default_rng(13).normal(size=(sum(n), 3))
    prm = mwlib.mw_params_default()
    prm.lambda_, prm.epsilon, prm.sigma = 21.0, 6.189 * 1.05, 2.3925 * 1.05
    po = orc.params(**{"lambda": 21.0, "epsilon": 6.189 * 1.05, "sigma": 2.3925 * 1.05})
    gx, gt = _gpu_vjp(mwlib, torch, n, np.array(boxes), np.concatenate(xs), w, prm)
    off = 0
    for b in range(3):
        gx_ref, gt_ref = orc.force_vjp(xs[b], boxes[b], w[off:off + n[b]], po)
        assert _rel_err_rows(gx[off:off + n[b]], gx_ref) <= G_TOL
        _check_theta(orc, xs[b], boxes[b], w[off:off + n[b]], gt[b], gt_ref, po)
        off += n[b]


def test_autograd_force_matching_step(mwlib, orc):
    """torch.autograd over the C ABI: d(loss)/d(x, theta) for a force-matching
    loss equals the oracle's chain rule."""
    torch = pytest.importorskip("torch")
    from paper_0809_2811_gb300 import torch_ops
    x, box = I.jittered_box(512, 1.0, 0.2, 700)
    x = I.snap_to_grid(x, box)
    f_target = orc.energy_forces(x, box)["forces"]  # the paper's parameters
    theta0 = [21.0, 6.189 * 1.05, 2.3925 * 1.05]
    ff = torch_ops.ForceField(len(x), box)
    try:
        xt = torch.tensor(x, device="cuda", requires_grad=True)
        th = torch.tensor(theta0, dtype=torch.float64, device="cuda", requires_grad=True)
        f = ff.forces(xt, th)
        loss = torch_ops.force_matching_loss(f, torch.tensor(f_target, device="cuda"))
        loss.backward()
        gx = xt.grad.cpu().numpy()
        gth = th.grad.cpu().numpy()
    finally:
        ff.close()
    po = orc.params(**{"lambda": theta0[0], "epsilon": theta0[1], "sigma": theta0[2]})
    f_cur = orc.energy_forces(x, box, po)["forces"]
    w = 2.0 * (f_cur - f_target) / f_cur.size
    gx_ref, gt_ref = orc.force_vjp(x, box, w, po)
    assert _rel_err_rows(gx, gx_ref) <= G_TOL
    _check_theta(orc, x, box, w, gth, gt_ref, po)
