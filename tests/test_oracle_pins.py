"""Pins of the FP64 oracle against facts other than itself (CPU only).

Each test checks the oracle against something the paper or the mathematics
fixes: closed-form eigenpairs, hand-derived worked examples, special cases
that reduce to textbook routines (LAPACK eigh, Kronecker products), the
Eq. 4 == Eq. 7 identity between two independent routines, brute force on
tiny inputs, Perron-Frobenius non-negativity, symmetry, and finite
differences for the adjoint.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import conv_form, dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
# sigma with g(d) = 2^{-d^2}: exp(-d^2 / (2 sigma^2)) = exp(-d^2 ln 2)
SIGMA_DYADIC = math.sqrt(1.0 / (2.0 * math.log(2.0)))


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# --------------------------------------------------------------------- taps
def test_taps_dyadic_values():
    """G of Eq. 1 at sigma^2 = 1/(2 ln 2) is 2^{-d^2}: 1, 1/2, 1/16, 1/512."""
    g = oracle.taps(3, SIGMA_DYADIC)
    np.testing.assert_allclose(g, [1 / 512, 1 / 16, 1 / 2, 1, 1 / 2, 1 / 16, 1 / 512],
                               rtol=1e-14)


# ------------------------------------------------------- worked 2-voxel case
def test_two_voxel_worked_example():
    """Hand-derived Eq. 2 / Eq. 4 example (tests/golden/two_voxel.json)."""
    with open(os.path.join(GOLDEN, "two_voxel.json")) as fh:
        gd = json.load(fh)
    shape = tuple(gd["shape"])
    s = np.array(gd["s"]).reshape(shape)
    sp = oracle.unary(s, gd["p"])
    np.testing.assert_allclose(sp.ravel(), [2.0, 0.5], rtol=1e-15)
    f = np.array(gd["f"]).reshape(shape)
    x = np.array(gd["x"]).reshape(shape)
    sig = (1.0, 1.0, SIGMA_DYADIC)
    y = oracle.apply_M(sp, f, x, gd["radii"], sig, gd["alpha"])
    np.testing.assert_allclose(y.ravel(), gd["y"], rtol=1e-15)
    # power iteration converges to the 2x2 textbook eigenvalue 17/8 + sqrt(234)/8
    out = oracle.power_iterate(sp, f, x, 200, gd["radii"], sig, gd["alpha"])
    lam = 17 / 8 + math.sqrt(234) / 8
    assert abs(out["rayleigh"][-1] - lam) < 1e-13 * lam
    assert out["residual"][-1] < 1e-12
    # residual and Rayleigh of step 0 from the hand-derived y = (19/4, 7/8)
    r0 = (1 * 4.75 + 2 * 0.875) / 5.0
    rho0 = math.hypot(4.75 - r0 * 1, 0.875 - r0 * 2) / math.sqrt(5.0)
    assert abs(out["rayleigh"][0] - r0) < 1e-15 and abs(out["residual"][0] - rho0) < 1e-15
    assert abs(out["norms"][0] - math.hypot(4.75, 0.875)) < 1e-14


def test_two_voxel_sign_and_alpha_terms():
    """Plausible mistakes (sign of the alpha term, f_i+f_j, missing square)
    change y of the worked example; check a second point with f far apart."""
    shape = (1, 1, 2)
    sp = np.array([1.0, 1.0]).reshape(shape)
    f = np.array([0.0, 0.5]).reshape(shape)
    x = np.array([1.0, 2.0]).reshape(shape)
    # M = [[1, 3/8], [3/8, 1]]
    y = oracle.apply_M(sp, f, x, (0, 0, 1), (1, 1, SIGMA_DYADIC), 1.0)
    np.testing.assert_allclose(y.ravel(), [1.75, 2.375], rtol=1e-15)
    # alpha = 2: 1 - 2/4 = 1/2, off-diagonal 1/4
    y = oracle.apply_M(sp, f, x, (0, 0, 1), (1, 1, SIGMA_DYADIC), 2.0)
    np.testing.assert_allclose(y.ravel(), [1.5, 2.25], rtol=1e-15)


# ----------------------------------------------- closed form: Kronecker sines
def _tridiag_eig(n, g):
    """Principal eigenpair of the n x n Toeplitz tridiagonal [g, 1, g]:
    u(i) = sin(pi (i+1)/(n+1)), lambda = 1 + 2 g cos(pi/(n+1))."""
    i = np.arange(n)
    u = np.sin(np.pi * (i + 1) / (n + 1))
    return 1 + 2 * g * math.cos(math.pi / (n + 1)), u / np.linalg.norm(u)


@pytest.mark.parametrize("shape", [(4, 5, 6), (3, 7, 2), (1, 1, 9)])
def test_constant_feature_kronecker_closed_form(shape):
    """f == c, S = F: M = c^{2p} T_t (x) T_y (x) T_x with radius-1 Toeplitz
    factors [g, 1, g] (zero padding); its principal eigenpair is the product
    of the 1D sine eigenvectors, lambda = c^{2p} prod(1 + 2g cos(pi/(n+1)))."""
    c, p, alpha = 0.7, 0.1, 1.0
    s = np.full(shape, c)
    sp = oracle.unary(s, p)
    f = np.full(shape, c)
    sig = (0.9, 1.3, SIGMA_DYADIC)
    g = [math.exp(-1 / (2 * sig[0] ** 2)), math.exp(-1 / (2 * sig[1] ** 2)), 0.5]
    lam = c ** (2 * p)
    vecs = []
    for n_a, g_a in zip(shape, g):
        l_a, u_a = _tridiag_eig(n_a, g_a)
        lam *= l_a
        vecs.append(u_a)
    v = np.einsum("i,j,k->ijk", *vecs)
    # one application: M v = lambda v
    y = oracle.apply_M(sp, f, v, (1, 1, 1), sig, alpha)
    assert rel(y, lam * v) < 1e-14
    # iteration from a positive start converges to it
    x0 = np.ones(shape) + 0.1 * np.random.default_rng(0).random(shape)
    out = oracle.power_iterate(sp, f, x0, 400, (1, 1, 1), sig, alpha)
    assert rel(out["x"], v) < 1e-9
    assert abs(out["rayleigh"][-1] - lam) < 1e-12 * lam


def test_alpha_zero_is_D_G_D_kronecker():
    """alpha = 0: M = D (G_t (x) G_y (x) G_x) D with D = diag(sp) and each
    G_a the banded Toeplitz matrix of the 1D Gaussian (zero padding)."""
    shape, radii, sig = (3, 4, 5), (1, 2, 2), (1.0, 1.5, 0.8)
    rng = np.random.default_rng(1)
    sp = rng.random(shape)
    f = rng.random(shape)
    x = rng.standard_normal(shape)

    def toeplitz(n, r, s):
        d = np.arange(n)[:, None] - np.arange(n)[None, :]
        return np.where(np.abs(d) <= r, np.exp(-d.astype(float) ** 2 / (2 * s * s)), 0.0)

    G = np.kron(np.kron(toeplitz(shape[0], radii[0], sig[0]), toeplitz(shape[1], radii[1], sig[1])),
                toeplitz(shape[2], radii[2], sig[2]))
    D = np.diag(sp.ravel())
    y_ref = D @ G @ D @ x.ravel()
    y = oracle.apply_M(sp, f, x, radii, sig, 0.0)
    assert rel(y, y_ref) < 1e-14


# ----------------------------------------------------------- special cases
def test_single_voxel():
    """1x1x1 volume: M = sp^2 (G(0) = 1), so lambda = sp^2, x stays 1."""
    sp = np.array([[[0.3]]])
    out = oracle.power_iterate(sp, np.array([[[0.9]]]), np.array([[[2.0]]]), 3,
                               (2, 5, 5), (1.5, 3.0, 3.0), 1.0)
    assert abs(out["rayleigh"][0] - 0.09) < 1e-16
    assert abs(out["x"].item() - 1.0) < 1e-15


def test_rt_zero_decouples_frames():
    """rt = 0: no temporal edges; x on frame 1 only maps to frame 1 only."""
    rng = np.random.default_rng(2)
    shape = (3, 6, 7)
    sp, f = rng.random(shape), rng.random(shape)
    x = np.zeros(shape)
    x[1] = rng.random(shape[1:])
    y = oracle.apply_M(sp, f, x, (0, 2, 2), (1.0, 1.0, 1.0), 0.5)
    assert np.all(y[0] == 0) and np.all(y[2] == 0) and np.any(y[1] != 0)


def test_zero_unary_voxels_vanish():
    """sp_i = 0 makes row i of M zero, so y_i = 0 after one step."""
    rng = np.random.default_rng(3)
    shape = (4, 6, 6)
    s = rng.random(shape)
    s[1, 2, :] = 0.0
    sp = oracle.unary(s, 0.1)
    assert np.all(sp[1, 2, :] == 0.0)
    y = oracle.apply_M(sp, rng.random(shape), rng.random(shape), (1, 2, 2), (1, 1, 1), 1.0)
    assert np.all(y[1, 2, :] == 0.0)


def test_unary_power_special_values():
    s = np.array([0.0, 1.0, 0.25, 4.0])
    np.testing.assert_array_equal(oracle.unary(s, 0.0), [1.0, 1.0, 1.0, 1.0])
    np.testing.assert_allclose(oracle.unary(s, 0.5), [0.0, 1.0, 0.5, 2.0], rtol=1e-15)


def test_zero_start_reports_zero_norm():
    shape = (2, 3, 3)
    out = oracle.power_iterate(np.ones(shape), np.zeros(shape), np.zeros(shape), 5,
                               (1, 1, 1), (1, 1, 1), 1.0)
    assert out["status"] == 1 and out["k_done"] == 0


# ---------------------------------------------- Eq. 4 == Eq. 7 (two routines)
@pytest.mark.parametrize("case", range(6))
def test_conv_form_equals_explicit(case):
    """Eq. 7 (x alpha) by direct 3D convolutions == Eq. 4 edge by edge, on
    random tiny volumes, random alpha, p in {0.1, 1}, odd radii, shapes
    smaller than the kernel."""
    rng = np.random.default_rng(100 + case)
    shape = tuple(int(v) for v in rng.integers(1, 9, size=3))
    radii = tuple(int(v) for v in rng.integers(0, 5, size=3))
    sig = tuple(float(v) for v in rng.uniform(0.5, 3.0, size=3))
    alpha = float(rng.uniform(0, 1))
    p = [0.1, 1.0][case % 2]
    sp = oracle.unary(rng.random(shape), p)
    f = rng.random(shape)
    x = rng.standard_normal(shape)
    gt, gy, gx = (oracle.taps(r, s) for r, s in zip(radii, sig))
    y_edge = oracle.apply_M(sp, f, x, radii, sig, alpha)
    y_conv = conv_form.apply_conv_form(sp, f, x, gt, gy, gx, alpha)
    assert rel(y_conv, y_edge) < 1e-13


def test_conv_form_equals_explicit_multichannel():
    """Eq. 9: the multi-channel result is the sum of per-channel Eq. 7."""
    rng = np.random.default_rng(7)
    shape, radii, sig = (5, 7, 9), (2, 3, 3), (1.5, 2.0, 2.0)
    sp = rng.random(shape)
    f = rng.random((2,) + shape)
    x = rng.random(shape)
    gt, gy, gx = (oracle.taps(r, s) for r, s in zip(radii, sig))
    y_edge = oracle.apply_M(sp, f, x, radii, sig, 0.7)
    y_conv = conv_form.apply_conv_form(sp, f, x, gt, gy, gx, 0.7)
    assert rel(y_conv, y_edge) < 1e-13
    y_sum = sum(oracle.apply_M(sp, f[c], x, radii, sig, 0.7) for c in range(2))
    assert rel(y_edge, y_sum) < 1e-14


def test_multichannel_special_cases():
    """Eq. 9 reduces to known operators: C identical channels give C times the
    single-channel M (same iterates, Rayleigh quotient times C); a channel that
    is zero everywhere adds sp_i sp_j G_ij, i.e. D G D with D = diag(sp)."""
    rng = np.random.default_rng(17)
    shape, radii, sig, alpha = (4, 6, 7), (1, 2, 2), (1.0, 1.5, 1.5), 0.8
    sp = oracle.unary(rng.random(shape), 0.1)
    f = rng.random(shape)
    x = rng.random(shape)
    y1 = oracle.apply_M(sp, f, x, radii, sig, alpha)
    for C in (2, 3):
        yC = oracle.apply_M(sp, np.stack([f] * C), x, radii, sig, alpha)
        assert rel(yC, C * y1) < 1e-14
        r1 = oracle.power_iterate(sp, f, x, 6, radii, sig, alpha)
        rC = oracle.power_iterate(sp, np.stack([f] * C), x, 6, radii, sig, alpha)
        assert rel(rC["x"], r1["x"]) < 1e-13
        np.testing.assert_allclose(rC["rayleigh"], C * np.asarray(r1["rayleigh"]), rtol=1e-12)
    y0 = oracle.apply_M(sp, np.stack([f, np.zeros(shape)]), x, radii, sig, alpha)
    ydgd = oracle.apply_M(sp, f, x, radii, sig, 0.0)          # alpha = 0: D G D x
    assert rel(y0, y1 + ydgd) < 1e-14


def test_binarized_reduces_to_plain_iteration():
    """k0 >= K: no projection, the plain power iteration."""
    from oracle import binarize
    rng = np.random.default_rng(23)
    shape, radii, sig = (3, 8, 9), (1, 2, 2), (1.0, 1.5, 1.5)
    sp = oracle.unary(rng.random(shape), 0.1)
    f = rng.random(shape)
    x0 = rng.random(shape)
    b = binarize.power_iterate_binarized(sp, f, x0, 6, radii, sig, 1.0, 6, 10.0, 0.5, 0.5)
    r = oracle.power_iterate(sp, f, x0, 6, radii, sig, 1.0)
    assert rel(b["x"], r["x"]) < 1e-13
    np.testing.assert_allclose(b["rayleigh"], r["rayleigh"], rtol=1e-13)


def test_binarized_beta_zero_restarts_from_uniform():
    """beta = 0 projects every voxel to 1/2 after every step from k0 on, so
    the last step starts from the uniform vector: x^K = M 1 / ||M 1||."""
    from oracle import binarize
    rng = np.random.default_rng(29)
    shape, radii, sig = (4, 7, 8), (1, 2, 2), (1.0, 1.5, 1.5)
    sp = oracle.unary(rng.random(shape), 0.1)
    f = rng.random(shape)
    x0 = rng.random(shape)
    K, k0 = 7, 3
    b = binarize.power_iterate_binarized(sp, f, x0, K, radii, sig, 1.0, k0, 0.0, 0.3, 0.5)
    r = oracle.power_iterate(sp, f, np.ones(shape), 1, radii, sig, 1.0)
    assert rel(b["x"], r["x"]) < 1e-13
    # and the Rayleigh quotients of steps k0 .. K-1 are those of the uniform vector
    r1 = oracle.power_iterate(sp, f, np.ones(shape), 1, radii, sig, 1.0)["rayleigh"][0]
    np.testing.assert_allclose(b["rayleigh"][k0:], r1, rtol=1e-13)


def test_binarized_two_voxel_by_hand():
    """The worked two-voxel example (M = [[4, 3/8], [3/8, 1/4]]) with one
    projection after step 1, values by hand: y1 = M (1, 2) = (19/4, 7/8),
    u = (1, 7/38); p = (s(beta (1 - tau)), s(beta (7/38 - tau))), s the
    logistic function; then y2 = M p / ||p|| and the mask at theta."""
    from oracle import binarize
    shape = (1, 1, 2)
    sp = np.array([2.0, 0.5]).reshape(shape)
    f = np.array([0.0, 0.5]).reshape(shape)
    x0 = np.array([1.0, 2.0]).reshape(shape)
    beta, tau = 4.0, 0.5
    out = binarize.power_iterate_binarized(sp, f, x0, 2, (0, 0, 1), (1, 1, SIGMA_DYADIC), 1.0, 1,
                                           beta, tau, 0.2)
    logistic = lambda t: 1.0 / (1.0 + math.exp(-t))
    p = np.array([logistic(beta * (1 - tau)), logistic(beta * (7 / 38 - tau))])
    p /= np.linalg.norm(p)
    y2 = np.array([4 * p[0] + 0.375 * p[1], 0.375 * p[0] + 0.25 * p[1]])
    np.testing.assert_allclose(out["x"].ravel(), y2 / np.linalg.norm(y2), rtol=1e-14)
    assert abs(out["rayleigh"][1] - float(p @ y2)) < 1e-14
    u2 = y2 / y2.max()
    np.testing.assert_array_equal(out["mask"].ravel(), (u2 >= 0.2).astype(np.uint8))


# -------------------------------------------- brute force + dense eigh (Fig. 3)
@pytest.mark.parametrize("shape", [(6, 10, 10), (2, 3, 4)])
def test_dense_matrix_and_eigh(shape):
    """Brute-force dense M (all voxel pairs) == edge loop; power iteration
    converges to LAPACK's principal eigenvector, which is >= 0
    (Perron-Frobenius, Sec. 3) because alpha * range(f)^2 <= 1."""
    rng = np.random.default_rng(11)
    radii, sig, alpha = (1, 2, 2), (1.0, 1.5, 1.5), 1.0
    sp = oracle.unary(rng.random(shape), 0.1)
    f = rng.random(shape)
    gt, gy, gx = (oracle.taps(r, s) for r, s in zip(radii, sig))
    M = dense.dense_M(sp, f, gt, gy, gx, alpha)
    assert np.array_equal(M, M.T)
    x = rng.standard_normal(shape)
    assert rel(oracle.apply_M(sp, f, x, radii, sig, alpha), M @ x.ravel()) < 1e-14
    lam, v = dense.principal_eigvec(M)
    assert np.all(v >= -1e-12)
    out = oracle.power_iterate(sp, f, f.copy(), 3000, radii, sig, alpha)
    assert rel(out["x"], v) < 1e-8
    assert abs(out["rayleigh"][-1] - lam) < 1e-10 * lam
    assert np.all(out["rayleigh"] <= lam * (1 + 1e-12))


def test_eigsh_4000_nodes():
    """10x20x20 = 4000 nodes (the graph size of the paper's timing, Sec. 4):
    the oracle's converged iterate matches ARPACK's principal eigenvector."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.linalg import eigsh
    shape, radii, sig, alpha = (10, 20, 20), (1, 2, 2), (1.0, 1.5, 1.5), 1.0
    rng = np.random.default_rng(12)
    sp = oracle.unary(rng.random(shape), 0.1)
    f = rng.random(shape)
    gt, gy, gx = (oracle.taps(r, s) for r, s in zip(radii, sig))
    M = dense.dense_M(sp, f, gt, gy, gx, alpha)
    lam, vec = eigsh(csr_matrix(M), k=1, which="LA", tol=1e-14)
    v = vec[:, 0] * np.sign(vec[:, 0].sum())
    out = oracle.power_iterate(sp, f, f.copy(), 4000, radii, sig, alpha)
    assert rel(out["x"], v) < 1e-7
    assert abs(out["rayleigh"][-1] - lam[0]) < 1e-10 * lam[0]


def test_exact_exponential_mode_matches_dense():
    """mode 1 (Eq. 1) == brute-force dense exact M; Eq. 2 is its first-order
    Taylor form, so the two differ by O(alpha^2) as alpha -> 0."""
    rng = np.random.default_rng(13)
    shape, radii, sig = (3, 5, 6), (1, 2, 2), (1.0, 1.5, 1.5)
    sp, f, x = rng.random(shape), rng.random(shape), rng.random(shape)
    gt, gy, gx = (oracle.taps(r, s) for r, s in zip(radii, sig))
    M1 = dense.dense_M(sp, f, gt, gy, gx, 0.8, exact=True)
    assert rel(oracle.apply_M(sp, f, x, radii, sig, 0.8, mode=1), M1 @ x.ravel()) < 1e-14
    errs = []
    for a in (1e-2, 1e-3):
        d = oracle.apply_M(sp, f, x, radii, sig, a, mode=1) - oracle.apply_M(sp, f, x, radii, sig, a)
        errs.append(np.abs(d).max())
    assert errs[1] < errs[0] / 50      # quadratic decay


# ------------------------------------------------------------- invariants
def test_symmetry_inner_products():
    """<u, M v> == <M u, v> (M symmetric, Sec. 3) for random u, v."""
    rng = np.random.default_rng(14)
    shape, radii, sig = (5, 8, 11), (2, 3, 4), (1.5, 2.0, 2.5)
    sp, f = rng.random(shape), rng.random(shape)
    u, v = rng.standard_normal(shape), rng.standard_normal(shape)
    a = np.vdot(u, oracle.apply_M(sp, f, v, radii, sig, 0.9))
    b = np.vdot(oracle.apply_M(sp, f, u, radii, sig, 0.9), v)
    assert abs(a - b) < 1e-12 * abs(a)


def test_nonnegative_iterates():
    """From x0 >= 0 every iterate stays >= 0 when alpha range(f)^2 <= 1."""
    rng = np.random.default_rng(15)
    shape = (6, 12, 14)
    sp = oracle.unary(rng.random(shape), 0.1)
    f = rng.random(shape)
    out = oracle.power_iterate(sp, f, f.copy(), 8, (2, 3, 3), (1.5, 2, 2), 1.0, keep=True)
    assert np.all(out["xs"] >= 0)


def test_sampled_outputs_match_full():
    rng = np.random.default_rng(16)
    shape, radii, sig = (4, 9, 10), (1, 3, 3), (1.5, 2, 2)
    sp, f, x = rng.random(shape), rng.random(shape), rng.random(shape)
    y = oracle.apply_M(sp, f, x, radii, sig, 1.0)
    idx = rng.integers(0, y.size, 50)
    np.testing.assert_array_equal(oracle.apply_M_at(sp, f, x, radii, sig, 1.0, idx), y.ravel()[idx])


# ---------------------------------------------------------------- adjoint
def _loss(sp, f, x0, K, radii, sig, alpha, target):
    return float(np.vdot(target, oracle.power_iterate(sp, f, x0, K, radii, sig, alpha)["x"]))


def test_adjoint_matches_finite_differences():
    """Central FD in FP64 along random directions vs the oracle's reverse
    mode, for L = sum(target * x^K)."""
    rng = np.random.default_rng(17)
    shape, radii, sig, alpha, K = (4, 6, 7), (1, 2, 2), (1.0, 1.5, 1.5), 1.0, 6
    sp = 0.5 + 0.5 * rng.random(shape)
    f = rng.random(shape)
    x0 = rng.random(shape)
    target = (rng.random(shape) > 0.5).astype(float)
    g_x0, g_sp, g_f, _ = oracle.adjoint(sp, f, x0, K, radii, sig, alpha, target)
    h = 1e-6
    for which, grad in (("x0", g_x0), ("sp", g_sp), ("f", g_f)):
        for _ in range(3):
            v = rng.standard_normal(shape)
            args = dict(sp=sp, f=f, x0=x0)
            ap, am = dict(args), dict(args)
            ap[which] = args[which] + h * v
            am[which] = args[which] - h * v
            fd = (_loss(ap["sp"], ap["f"], ap["x0"], K, radii, sig, alpha, target)
                  - _loss(am["sp"], am["f"], am["x0"], K, radii, sig, alpha, target)) / (2 * h)
            an = float(np.vdot(grad, v))
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (which, fd, an)


def test_adjoint_scale_invariance():
    """x^K does not depend on the scale of x0, so x0 . dL/dx0 = 0."""
    rng = np.random.default_rng(18)
    shape = (3, 8, 8)
    sp, f, x0 = rng.random(shape), rng.random(shape), rng.random(shape)
    g_x0, _, _, _ = oracle.adjoint(sp, f, x0, 5, (1, 2, 2), (1, 1.5, 1.5), 1.0,
                                   rng.random(shape))
    assert abs(np.vdot(x0, g_x0)) < 1e-12 * np.linalg.norm(x0) * np.linalg.norm(g_x0)


def test_storage_rounding():
    """bf16 round-to-nearest-even of known values."""
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 3.14159265], np.float32)
    np.testing.assert_array_equal(oracle.to_storage(a, "bf16")[:3],
                                  [1.0, 1.0, 1.0 + 2 ** -6])
    assert abs(oracle.to_storage(a, "bf16")[3] - 3.140625) == 0
