"""GPU parity of the collision penalty (forward, hand-written backward, autograd).

The oracle's fp64 loss and analytic gradient (pinned in test_oracle_pins.py by
central differences and by the closed-form point-to-line gradient) are the
reference.  Gradients must agree to 1e-4 relative, both norm-wise and
elementwise against max(|g_ref|, 1e-3 |g_ref|_inf), the largest component
taken over the whole gradient (all vertices, or all poses).  The library takes
tau as a float32, so the oracle is given that same float32 value.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from paper_2007_15385_gb300 import binding as B
from paper_2007_15385_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    yield


def _to(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _rel_ok(got, want, tol=1e-4):
    got = np.asarray(got, float).ravel()
    want = np.asarray(want, float).ravel()
    nrm = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)
    floor = 1e-3 * np.abs(want).max()
    elem = np.abs(got - want) <= tol * np.maximum(np.abs(want), floor)
    bad = np.flatnonzero(~elem)[:6]
    detail = ", ".join("[%d] %.9g vs %.9g" % (i, got[i], want[i]) for i in bad)
    return nrm <= tol and elem.all(), nrm, "%d (%s)" % (int((~elem).sum()), detail)


def _tau32(tau):
    return float(np.float32(tau))


def _oracle(v, P, q, tau):
    return oracle.penalty(v.astype(np.float64), P.astype(np.float64), q.astype(np.float64), _tau32(tau))


def _oracle_threads(v, P, q, tau):
    """oracle.penalty over blocks of poses on every host core: the loss and
    the vertex gradient add over poses, the pose rows are the blocks' own."""
    qd = q.astype(np.float64)
    blocks = np.array_split(np.arange(len(P)), min(len(P), os.cpu_count() or 1))
    with ThreadPoolExecutor(len(blocks)) as ex:
        parts = list(ex.map(lambda b: oracle.penalty(v.astype(np.float64), P[b].astype(np.float64), qd,
                                                     _tau32(tau)), blocks))
    loss = sum(r[0] for r in parts)
    gv = sum(r[1] for r in parts)
    gp = np.concatenate([r[2] for r in parts])
    return loss, gv, gp


def _case(m=8192, poses=12, seed=40):
    w = wl.footprint_trajectory(seed=seed, m=m, num_poses=poses)
    return w.vertices, w.extra["poses"], w.points, w.extra["tau"]


@pytest.mark.parametrize("cull", [False, True])
def test_penalty_loss_and_gradients_match_fp64_reference(cull):
    v, P, q, tau = _case()
    loss = B.pip_penalty_forward(_to(v), _to(P), _to(q), tau, cull=cull).item()
    gv, gp = B.pip_penalty_backward(_to(v), _to(P), _to(q), tau, cull=cull)
    ref_loss, ref_gv, ref_gp = _oracle(v, P, q, tau)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    ok, nrm, bad = _rel_ok(gv.cpu().numpy(), ref_gv)
    assert ok, "vertex gradient: norm-wise %.2e, %s elements off" % (nrm, bad)
    ok, nrm, bad = _rel_ok(gp.cpu().numpy(), ref_gp)
    assert ok, "pose gradient: norm-wise %.2e, %s elements off" % (nrm, bad)


@pytest.mark.parametrize("cull", [False, True])
@pytest.mark.parametrize("n", [4, 7, 16, 20, 40])
def test_penalty_other_edge_counts(n, cull):
    """Register variants for up to 4, 8 and 16 edges and the shared-memory
    variant above 16, each against the oracle, with and without the cull."""
    w = wl.footprint_trajectory(seed=45 + n, m=6000, num_poses=7, n=n)
    v, P, q, tau = w.vertices, w.extra["poses"], w.points, w.extra["tau"]
    loss = B.pip_penalty_forward(_to(v), _to(P), _to(q), tau, cull=cull).item()
    gv, gp = B.pip_penalty_backward(_to(v), _to(P), _to(q), tau, cull=cull)
    ref_loss, ref_gv, ref_gp = _oracle(v, P, q, tau)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    ok, nrm, bad = _rel_ok(gv.cpu().numpy(), ref_gv)
    assert ok, "n=%d vertex gradient: norm-wise %.2e, %s elements off" % (n, nrm, bad)
    ok, nrm, bad = _rel_ok(gp.cpu().numpy(), ref_gp)
    assert ok, "n=%d pose gradient: norm-wise %.2e, %s elements off" % (n, nrm, bad)


def test_penalty_gradient_against_central_differences_of_fp64_loss():
    v, P, q, tau = _case(m=2048, poses=4, seed=41)
    gv, gp = B.pip_penalty_backward(_to(v), _to(P), _to(q), tau)
    gv = gv.cpu().numpy()
    gp = gp.cpu().numpy()
    vd, Pd, qd = v.astype(np.float64), P.astype(np.float64), q.astype(np.float64)
    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(8):
        i, d = int(rng.integers(len(v))), int(rng.integers(2))
        vp, vm = vd.copy(), vd.copy()
        vp[i, d] += h
        vm[i, d] -= h
        fd = (oracle.penalty_loss(vp, Pd, qd, _tau32(tau)) - oracle.penalty_loss(vm, Pd, qd, _tau32(tau))) / (2 * h)
        assert gv[i, d] == pytest.approx(fd, rel=1e-4, abs=1e-4 * np.abs(gv).max())
    for j in range(len(P)):
        for d in range(3):
            pp, pm = Pd.copy(), Pd.copy()
            pp[j, d] += h
            pm[j, d] -= h
            fd = (oracle.penalty_loss(vd, pp, qd, _tau32(tau)) - oracle.penalty_loss(vd, pm, qd, _tau32(tau))) / (2 * h)
            assert gp[j, d] == pytest.approx(fd, rel=1e-4, abs=1e-4 * np.abs(gp).max())


@pytest.mark.parametrize("cull", [False, True])
def test_penalty_autograd_function(cull):
    v, P, q, tau = _case(m=4096, poses=6, seed=42)
    vt = _to(v).requires_grad_(True)
    pt = _to(P).requires_grad_(True)
    loss = B.collision_penalty(vt, pt, _to(q), tau, cull=cull)
    (3.0 * loss).backward()
    gv, gp = B.pip_penalty_backward(_to(v), _to(P), _to(q), tau, cull=cull)
    np.testing.assert_allclose(vt.grad.cpu().numpy(), 3.0 * gv.cpu().numpy(), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(pt.grad.cpu().numpy(), 3.0 * gp.cpu().numpy(), rtol=1e-6, atol=1e-6)


def test_penalty_translation_invariance_on_gpu():
    v, P, q, tau = _case(m=4096, poses=5, seed=43)
    l0 = B.pip_penalty_forward(_to(v), _to(P), _to(q), tau).item()
    shift = np.array([4.0, -2.0], np.float32)
    P2 = P.copy()
    P2[:, :2] += shift
    l1 = B.pip_penalty_forward(_to(v), _to(P2), _to(q + shift), tau).item()
    assert l1 == pytest.approx(l0, rel=1e-5)


@pytest.mark.parametrize("cull", [False, True])
def test_penalty_empty_points_and_invalid_footprint(cull):
    v, P, q, tau = _case(m=16, poses=2, seed=44)
    assert B.pip_penalty_forward(_to(v), _to(P), _to(q[:0]), tau, cull=cull).item() == 0.0
    bad = np.array([[0, 0], [2, 0], [1, 0.2], [2, 2], [0, 2]], np.float32)  # non-convex
    assert B.pip_penalty_forward(_to(bad), _to(P), _to(q), tau, cull=cull).item() == 0.0
    gv, gp = B.pip_penalty_backward(_to(bad), _to(P), _to(q), tau, cull=cull)
    assert not gv.cpu().numpy().any() and not gp.cpu().numpy().any()


def test_penalty_cull_of_points_all_far_away():
    """Every point hundreds of tau beyond the footprint: every term and
    gradient is exactly 0 in float32, with the cull (nothing kept) and
    without; one point near a pose keeps the loss and gradient equal to the
    full pass's and the oracle's."""
    v, P, q, tau = _case(m=4000, poses=3, seed=46)
    far = (q + np.float32(1000.0)).astype(np.float32)
    for cull in (False, True):
        assert B.pip_penalty_forward(_to(v), _to(P), _to(far), tau, cull=cull).item() == 0.0
        gv, gp = B.pip_penalty_backward(_to(v), _to(P), _to(far), tau, cull=cull)
        assert not gv.cpu().numpy().any() and not gp.cpu().numpy().any()
    far[1234] = P[1, :2] + np.float32(0.5)
    ref_loss, ref_gv, ref_gp = _oracle(v, P, far, tau)
    for cull in (False, True):
        loss = B.pip_penalty_forward(_to(v), _to(P), _to(far), tau, cull=cull).item()
        gv, gp = B.pip_penalty_backward(_to(v), _to(P), _to(far), tau, cull=cull)
        assert loss == pytest.approx(ref_loss, rel=1e-5)
        ok, nrm, bad = _rel_ok(gv.cpu().numpy(), ref_gv)
        assert ok, "cull=%s vertex gradient: norm-wise %.2e, %s elements off" % (cull, nrm, bad)
        ok, nrm, bad = _rel_ok(gp.cpu().numpy(), ref_gp)
        assert ok, "cull=%s pose gradient: norm-wise %.2e, %s elements off" % (cull, nrm, bad)


def test_penalty_full_size_every_gradient():
    """The full workload (256 poses x 2^20 points, the benchmark's launch
    shape): the loss, all 24 vertex gradients and all 768 pose gradients
    against the oracle run over pose blocks on every host core."""
    w = wl.footprint_trajectory()
    v, P, q, tau = w.vertices, w.extra["poses"], w.points, w.extra["tau"]
    ref_loss, ref_gv, ref_gp = _oracle_threads(v, P, q, tau)
    for cull in (False, True):
        loss = B.pip_penalty_forward(_to(v), _to(P), _to(q), tau, cull=cull).item()
        gv, gp = B.pip_penalty_backward(_to(v), _to(P), _to(q), tau, cull=cull)
        assert loss == pytest.approx(ref_loss, rel=1e-5)
        ok, nrm, bad = _rel_ok(gv.cpu().numpy(), ref_gv)
        assert ok, "cull=%s vertex gradient: norm-wise %.2e, %s of 24 elements off" % (cull, nrm, bad)
        ok, nrm, bad = _rel_ok(gp.cpu().numpy(), ref_gp)
        assert ok, "cull=%s pose gradient: norm-wise %.2e, %s of 768 elements off" % (cull, nrm, bad)


@pytest.mark.parametrize("cull", [False, True])
@pytest.mark.parametrize("n", [12, 20])
def test_penalty_every_pair_near_the_footprint(n, cull):
    """Poses near the origin and points within 3 m of it: every (pose, point)
    pair has a nonzero gradient, so every warp's queue fills on every step
    (the benchmark's trajectory has ~6 % such pairs)."""
    w = wl.footprint_trajectory(seed=60 + n, m=16, num_poses=2, n=n)
    rng = np.random.default_rng(61)
    P = np.stack([rng.uniform(-0.3, 0.3, 6), rng.uniform(-0.3, 0.3, 6), rng.uniform(-3.1, 3.1, 6)],
                 axis=1).astype(np.float32)
    q = rng.uniform(-3.0, 3.0, size=(5003, 2)).astype(np.float32)
    v, tau = w.vertices, w.extra["tau"]
    loss = B.pip_penalty_forward(_to(v), _to(P), _to(q), tau, cull=cull).item()
    gv, gp = B.pip_penalty_backward(_to(v), _to(P), _to(q), tau, cull=cull)
    ref_loss, ref_gv, ref_gp = _oracle(v, P, q, tau)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    ok, nrm, bad = _rel_ok(gv.cpu().numpy(), ref_gv)
    assert ok, "n=%d vertex gradient: norm-wise %.2e, %s elements off" % (n, nrm, bad)
    ok, nrm, bad = _rel_ok(gp.cpu().numpy(), ref_gp)
    assert ok, "n=%d pose gradient: norm-wise %.2e, %s elements off" % (n, nrm, bad)
