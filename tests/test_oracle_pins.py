"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test ties one step of the projector, or the whole operator, to a
library routine, a closed form, a hand-worked example or an exact
invariant, so that a dropped term, a flipped sign, a transposed operand or
a wrong padding rule in the oracle fails at least one of them:

  rotation      -> scipy.ndimage.affine_transform (order 1, zero fill) and
                   exact lattice permutations at multiples of 90 degrees
  attenuation   -> closed form for a uniform map, Eq. (1)
  PSF blur      -> scipy.ndimage.convolve(mode="nearest") and a hand-worked
                   1D example (tests/golden/conv_replicate_1d.txt)
  PSF factors   -> the outer product written index by index, and a blur with
                   the built stack == scipy convolve1d along i, then along k
  forward A     -> composition of the library routines above (Algorithm 1),
                   line sums for a delta PSF without attenuation
  back A'       -> dense-matrix transpose of A (the paper's Section III-A
                   adjoint experiment, 336 x 384) and Eq. (2)
  EM            -> count preservation, fixed point, monotone likelihood
  3-pass rotation -> shear algebra, scipy order-1 resampling per pass, lattice
                   permutations, a blob turned by +theta, exact mass
                   conservation, dense transpose (reading R13)
"""
import os

import numpy as np
import pytest
from scipy import ndimage

import oracle
from paper_2301_09710_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ rotation
def _scipy_rotate(img, theta):
    """Bilinear rotation by the library: out[j,i] = img at (ys, xs), zero outside."""
    n = img.shape[0]
    c = 0.5 * (n - 1)
    ct, st = np.cos(theta), np.sin(theta)
    # (ys, xs) = M @ (j, i) + off, from xs = c + ct(i-c) + st(j-c), ys = c - st(i-c) + ct(j-c)
    m = np.array([[ct, -st], [st, ct]])
    off = np.array([c - ct * c + st * c, c - st * c - ct * c])
    return ndimage.affine_transform(img, m, offset=off, order=1, mode="grid-constant", cval=0.0)


@pytest.mark.parametrize("theta", [0.1, 0.7853981633974483, 1.0, 2.5, 4.0, 5.9])
@pytest.mark.parametrize("n", [7, 16])
def test_rotation_matches_scipy_bilinear(n, theta):
    rng = np.random.default_rng(1)
    img = rng.uniform(-1, 1, (n, n))
    got = oracle.rotate_slice(img, theta)
    ref = _scipy_rotate(img, theta)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("quarter", [0, 1, 2, 3])
def test_rotation_quarter_turns_are_lattice_permutations(quarter):
    rng = np.random.default_rng(2)
    img = rng.uniform(0, 1, (9, 9))
    got = oracle.rotate_slice(img, quarter * np.pi / 2)
    # content turns by +theta: at 90 degrees out(i, j) = in(j, n-1-i)
    np.testing.assert_array_equal(got, np.rot90(img, -quarter))


@pytest.mark.parametrize("theta", [0.3, 1.7, 3.0])
def test_rotation_adjoint_is_transpose_not_inverse_rotation(theta):
    n = 8
    R = np.stack([oracle.rotate_slice(e.reshape(n, n), theta).ravel() for e in np.eye(n * n)], axis=1)
    Rt = np.stack([oracle.rotate_adjoint_slice(e.reshape(n, n), theta).ravel() for e in np.eye(n * n)], axis=1)
    np.testing.assert_allclose(Rt, R.T, rtol=0, atol=1e-15)
    # Section II-A: rotating by -theta is not the adjoint of a discrete rotation.
    Rminus = np.stack([oracle.rotate_slice(e.reshape(n, n), -theta).ravel() for e in np.eye(n * n)], axis=1)
    assert np.linalg.norm(Rminus - R.T) > 1e-2 * np.linalg.norm(R)


# ------------------------------------------------------------------ attenuation
def test_attenuation_uniform_closed_form():
    nx, ny, nz, mu0, dy = 5, 11, 3, 0.07, 4.8
    mu = np.full((nz, ny, nx), mu0)
    got = oracle.attenuation(mu, dy)
    j = np.arange(ny)
    want = np.exp(-dy * mu0 * (0.5 + (ny - 1 - j)))
    np.testing.assert_allclose(got, np.broadcast_to(want[None, :, None], got.shape), rtol=1e-14)


def test_attenuation_single_plane_and_step():
    # only plane s = 6 attenuates: planes j < 6 see the full mu, j = 6 half, j > 6 none
    nx, ny, nz, dy = 2, 10, 1, 2.0
    mu = np.zeros((nz, ny, nx))
    mu[:, 6, :] = 0.3
    got = oracle.attenuation(mu, dy)[0, :, 0]
    want = np.where(np.arange(ny) < 6, np.exp(-dy * 0.3), 1.0)
    want[6] = np.exp(-dy * 0.15)
    np.testing.assert_allclose(got, want, rtol=1e-15)


# ------------------------------------------------------------------ PSF blur
def test_conv_matches_scipy_convolve_nearest():
    rng = np.random.default_rng(3)
    w = rng.uniform(0, 1, (13, 17))  # (nz, nx)
    p = rng.uniform(0, 1, (7, 5))    # (pz, px), deliberately non-symmetric
    got = oracle.conv_plane(w, p)
    ref = ndimage.convolve(w, p, mode="nearest")
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=0)


def test_conv_psf_wider_than_plane_matches_scipy():
    rng = np.random.default_rng(4)
    w = rng.uniform(0, 1, (3, 4))
    p = rng.uniform(0, 1, (9, 11))
    np.testing.assert_allclose(oracle.conv_plane(w, p), ndimage.convolve(w, p, mode="nearest"), rtol=1e-13)


def _asymmetric_factors(rng, nvp, ny, px, pz):
    """Separable factors with no symmetry, px != pz, different per depth and view."""
    fx = rng.uniform(0.1, 1.0, (nvp, ny, px)) * np.linspace(1.0, 2.0, px)
    fz = rng.uniform(0.1, 1.0, (nvp, ny, pz)) * np.linspace(2.0, 0.5, pz)
    return fx.astype(np.float32), fz.astype(np.float32)


def test_psf_from_factors_is_the_outer_product_by_index():
    """p(a,b,j,l) = fx(a,j,l) fz(b,j,l), written out index by index: a swap of the
    factors, of a and b, or of the depth / view axes changes the stack."""
    rng = np.random.default_rng(21)
    nvp, ny, px, pz = 3, 4, 5, 3
    fx, fz = _asymmetric_factors(rng, nvp, ny, px, pz)
    got = oracle.psf_from_factors(fx, fz)
    assert got.shape == (nvp, ny, pz, px)
    for l in range(nvp):
        for j in range(ny):
            for b in range(pz):
                for a in range(px):
                    assert got[l, j, b, a] == np.float64(fx[l, j, a]) * np.float64(fz[l, j, b])


def test_psf_from_factors_blur_equals_two_1d_convolutions():
    """A blur with the stack built from (fx, fz) equals scipy's 1D replicate-padded
    convolution along i with fx followed by the one along k with fz (Section II-A:
    replicate padding acts on each axis on its own, so the separable blur
    factorises), for every depth and view of the stack."""
    rng = np.random.default_rng(22)
    nvp, ny, px, pz = 2, 3, 7, 5
    fx, fz = _asymmetric_factors(rng, nvp, ny, px, pz)
    psf = oracle.psf_from_factors(fx, fz)
    w = rng.uniform(0, 1, (9, 11))  # (nz, nx)
    for l in range(nvp):
        for j in range(ny):
            u = ndimage.convolve1d(w, fx[l, j].astype(np.float64), axis=1, mode="nearest")
            want = ndimage.convolve1d(u, fz[l, j].astype(np.float64), axis=0, mode="nearest")
            np.testing.assert_allclose(oracle.conv_plane(w, psf[l, j]), want, rtol=1e-13, atol=0)


def _golden_conv():
    rows = []
    with open(os.path.join(GOLDEN, "conv_replicate_1d.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("psf"):
                psf = np.array([float(t) for t in line.split()[1:]])
            else:
                rows.append([float(t) for t in line.split()])
    return psf, np.array(rows)


def test_conv_replicate_hand_worked_1d_and_its_transpose():
    psf, M = _golden_conv()
    n = M.shape[0]
    p = psf[None, :]
    F = np.stack([oracle.conv_plane(e[None, :], p)[0] for e in np.eye(n)], axis=1)
    B = np.stack([oracle.conv_adjoint_plane(e[None, :], p)[0] for e in np.eye(n)], axis=1)
    np.testing.assert_array_equal(F, M)
    np.testing.assert_array_equal(B, M.T)


# ------------------------------------------------------------------ forward operator
def _library_forward(x, mu, psf, dy, angles):
    """Algorithm 1 composed from library routines only (scipy / numpy)."""
    nz, ny, nx = x.shape
    out = np.zeros((len(angles), nz, nx))
    for l, th in enumerate(angles):
        xr = np.stack([_scipy_rotate(x[k].astype(np.float64), th) for k in range(nz)])
        mr = np.stack([_scipy_rotate(mu[k].astype(np.float64), th) for k in range(nz)])
        # S(j) = mu(j)/2 + sum_{s>j} mu(s): reverse cumulative sum along j
        tail = np.flip(np.cumsum(np.flip(mr, axis=1), axis=1), axis=1) - mr
        mbar = np.exp(-dy * (0.5 * mr + tail))
        w = xr * mbar
        p = psf[0 if psf.shape[0] == 1 else l]
        for j in range(ny):
            out[l] += ndimage.convolve(w[:, j, :], p[j].astype(np.float64), mode="nearest")
    return out


def test_forward_matches_library_composition():
    prob = synthetic.random_problem(5, nx=12, nz=6, nview=5, px=5, pz=3, nview_psf=5)
    angles = np.array([0.0, 0.4, 1.3, 2.9, 5.0])
    got = oracle.forward(prob.x, prob.mu, prob.psf, 1.7, angles)
    want = _library_forward(prob.x, prob.mu, prob.psf, 1.7, angles)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)


def _delta_psf(ny, px, pz, nview_psf=1):
    p = np.zeros((nview_psf, ny, pz, px))
    p[:, :, (pz - 1) // 2, (px - 1) // 2] = 1.0
    return p


def test_forward_theta0_no_attenuation_delta_psf_is_line_sum():
    rng = np.random.default_rng(6)
    x = rng.uniform(0, 1, (4, 9, 9))
    v = oracle.forward(x, np.zeros_like(x), _delta_psf(9, 3, 5), 1.0, [0.0])
    np.testing.assert_allclose(v[0], x.sum(axis=1), rtol=1e-14)


def test_forward_quarter_turns_are_rotated_line_sums():
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, (3, 8, 8))
    angles = np.array([0, 1, 2, 3]) * np.pi / 2
    v = oracle.forward(x, np.zeros_like(x), _delta_psf(8, 1, 1), 1.0, angles)
    for q in range(4):
        want = np.stack([np.rot90(x[k], -q).sum(axis=0) for k in range(3)])
        np.testing.assert_allclose(v[q], want, rtol=1e-14)


def test_forward_uniform_slice_survives_any_unit_sum_psf():
    # replicate padding keeps a uniform plane uniform: v = ny * value when theta = 0, mu = 0
    n, nz = 6, 4
    x = np.full((nz, n, n), 2.5)
    rng = np.random.default_rng(8)
    p = rng.uniform(0, 1, (1, n, 5, 7))
    p /= p.sum(axis=(2, 3), keepdims=True)
    v = oracle.forward(x, np.zeros_like(x), p, 1.0, [0.0])
    np.testing.assert_allclose(v, 2.5 * n, rtol=1e-14)


def test_forward_single_voxel_gives_scaled_psf_copy():
    n, nz, j0 = 16, 16, 5
    x = np.zeros((nz, n, n))
    x[8, j0, 7] = 1.0
    mu0, dy = 0.02, 3.0
    mu = np.full_like(x, mu0)
    rng = np.random.default_rng(9)
    p = rng.uniform(0, 1, (1, n, 5, 3))
    v = oracle.forward(x, mu, p, dy, [0.0])[0]
    scale = np.exp(-dy * mu0 * (0.5 + (n - 1 - j0)))
    want = np.zeros((nz, n))
    # true convolution: out(i,k) = p(i - 7 + cx, k - 8 + cz)
    for b in range(5):
        for a in range(3):
            want[8 + b - 2, 7 + a - 1] = p[0, j0, b, a]
    np.testing.assert_allclose(v, scale * want, rtol=1e-13, atol=1e-16)


def test_count_conservation_quarter_turns_and_approximate_otherwise():
    # support inside the inscribed circle and away from every edge the blur
    # reaches, so neither zero padding nor replicate padding touches it
    n, nz = 16, 5
    x = np.zeros((nz, n, n))
    rng = np.random.default_rng(10)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    inside = (ii - 7.5) ** 2 + (jj - 7.5) ** 2 < 4.5 ** 2
    x[1:nz - 1, inside] = rng.uniform(0, 1, (nz - 2, inside.sum()))
    p = rng.uniform(0, 1, (1, n, 3, 5))
    p /= p.sum(axis=(2, 3), keepdims=True)
    mu = np.zeros_like(x)
    v = oracle.forward(x, mu, p, 1.0, np.array([0, 1, 2, 3]) * np.pi / 2)
    np.testing.assert_allclose(v.sum(axis=(1, 2)), x.sum(), rtol=1e-13)
    v2 = oracle.forward(x, mu, p, 1.0, [0.3, 1.1, 2.2])
    np.testing.assert_allclose(v2.sum(axis=(1, 2)), x.sum(), rtol=1e-2)


def test_forward_is_linear():
    prob = synthetic.random_problem(11, nx=10, nz=4, nview=3, px=3, pz=3)
    ang = [0.2, 1.9, 4.4]
    rng = np.random.default_rng(11)
    x1 = prob.x.astype(np.float64)
    x2 = rng.uniform(0, 1, prob.x.shape)
    a, b = 0.7, -1.3
    lhs = oracle.forward(a * x1 + b * x2, prob.mu, prob.psf, 1.0, ang)
    rhs = a * oracle.forward(x1, prob.mu, prob.psf, 1.0, ang) + b * oracle.forward(x2, prob.mu, prob.psf, 1.0, ang)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------------ adjoint A'
def _dense(nx, nz, nview, mu, psf, dy, angles):
    ny = nx
    N, M = nx * ny * nz, nx * nz * nview
    A = np.empty((M, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        A[:, c] = oracle.forward(e.reshape(nz, ny, nx), mu, psf, dy, angles, nthreads=1).ravel()
    B = np.empty((N, M))
    for r in range(M):
        e = np.zeros(M)
        e[r] = 1.0
        B[:, r] = oracle.back(e.reshape(nview, nz, nx), mu, psf, dy, angles, nthreads=1).ravel()
    return A, B


@pytest.mark.parametrize("symmetric", [True, False])
def test_dense_adjoint_paper_shape(symmetric):
    # Section III-A: (8*6*7) x (8*8*6) system matrix, random non-negative mu and PSF
    for seed in range(3):
        prob = synthetic.random_problem(100 + seed, nx=8, nz=6, nview=7, px=3, pz=3, symmetric=symmetric, mu_scale=0.3)
        angles = oracle.default_angles(7)
        A, B = _dense(8, 6, 7, prob.mu, prob.psf, 1.0, angles)
        assert A.shape == (336, 384)
        err = np.linalg.norm(A.T - B) / np.linalg.norm(A)
        assert err < 1e-14, err


@pytest.mark.slow
def test_dense_adjoint_16x16x8_psf5():
    prob = synthetic.random_problem(12, nx=16, nz=8, nview=8, px=5, pz=5, nview_psf=8, mu_scale=0.2)
    A, B = _dense(16, 8, 8, prob.mu, prob.psf, 1.5, oracle.default_angles(8) + 0.1)
    assert np.linalg.norm(A.T - B) / np.linalg.norm(A) < 1e-14


def test_adjoint_identity_random():
    prob = synthetic.random_problem(13, nx=20, nz=9, nview=11, px=7, pz=5, nview_psf=11, mu_scale=0.1)
    rng = np.random.default_rng(13)
    y = rng.uniform(-1, 1, (11, 9, 20))
    ang = rng.uniform(0, 2 * np.pi, 11)
    Ax = oracle.forward(prob.x, prob.mu, prob.psf, 2.0, ang)
    Aty = oracle.back(y, prob.mu, prob.psf, 2.0, ang)
    lhs, rhs = np.vdot(Ax, y), np.vdot(prob.x.astype(np.float64), Aty)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_back_thread_count_invariant():
    prob = synthetic.random_problem(14, nx=10, nz=3, nview=7, px=3, pz=3)
    rng = np.random.default_rng(14)
    y = rng.uniform(0, 1, (7, 3, 10))
    ang = oracle.default_angles(7)
    a = oracle.back(y, prob.mu, prob.psf, 1.0, ang, nthreads=1)
    b = oracle.back(y, prob.mu, prob.psf, 1.0, ang, nthreads=3)
    np.testing.assert_array_equal(a, b)


# ------------------------------------------------------------------ EM
def _em_problem():
    prob = synthetic.config1(seed=0, nx=16, nz=6, nview=12, psf_size=5)
    psf = prob.full_psf()
    ang = oracle.default_angles(prob.nview)
    return prob, psf, ang


def test_em_preserves_counts_with_zero_background():
    prob, psf, ang = _em_problem()
    rng = np.random.default_rng(15)
    y = rng.poisson(5.0, (prob.nview, 6, 16)).astype(np.float64)
    s = oracle.sensitivity(prob.mu, psf, prob.dy, ang)
    x = np.ones((6, 16, 16))
    for _ in range(3):
        x = oracle.em_step(x, y, None, prob.mu, psf, prob.dy, ang, s=s)
        # sum_j s_j x_j^{k+1} = sum_i y_i when rbar = 0
        assert abs(np.sum(s * x) - y.sum()) <= 1e-11 * y.sum()
        assert np.all(x >= 0)


def test_em_fixed_point_at_truth():
    prob, psf, ang = _em_problem()
    xt = prob.x.astype(np.float64) + 0.1
    y = oracle.forward(xt, prob.mu, psf, prob.dy, ang)
    x1 = oracle.em_step(xt, y, None, prob.mu, psf, prob.dy, ang)
    np.testing.assert_allclose(x1, xt, rtol=1e-12)


def test_em_loglik_monotone_and_positive():
    prob, psf, ang = _em_problem()
    xt = prob.x.astype(np.float64)
    ybar = oracle.forward(xt, prob.mu, psf, prob.dy, ang)
    rbar = 0.1 * ybar.mean() * np.ones_like(ybar)
    y = np.random.default_rng(16).poisson(ybar + rbar).astype(np.float64)
    s = oracle.sensitivity(prob.mu, psf, prob.dy, ang)
    x = np.ones_like(xt)
    ll = [oracle.poisson_loglik(x, y, rbar, prob.mu, psf, prob.dy, ang)]
    for _ in range(5):
        x = oracle.em_step(x, y, rbar, prob.mu, psf, prob.dy, ang, s=s)
        assert np.all(x[s > 0] > 0)
        ll.append(oracle.poisson_loglik(x, y, rbar, prob.mu, psf, prob.dy, ang))
    assert all(b >= a - 1e-9 * abs(a) for a, b in zip(ll, ll[1:])), ll


# ------------------------------------------------------------------ regularised EM (Eqs. (7)-(8))
def test_em_reg_reduces_to_mlem_as_beta_vanishes():
    prob, psf, ang = _em_problem()
    rng = np.random.default_rng(17)
    y = rng.poisson(5.0, (prob.nview, 6, 16)).astype(np.float64)
    x = np.ones((6, 16, 16))
    u = rng.uniform(0, 2, x.shape)
    mlem = oracle.em_step(x, y, None, prob.mu, psf, prob.dy, ang)
    reg = oracle.em_step_reg(x, y, None, u, 1e-12, prob.mu, psf, prob.dy, ang)
    np.testing.assert_allclose(reg, mlem, rtol=1e-9)


def test_em_reg_solves_the_surrogate_quadratic():
    # the update is the non-negative root of beta x^2 + d x - x_k e = 0 with
    # d = A'1 - beta u and e = A'(y / (A x_k + rbar)) (the EM surrogate)
    prob, psf, ang = _em_problem()
    rng = np.random.default_rng(18)
    xk = rng.uniform(0.5, 2, (6, 16, 16))
    y = rng.poisson(8.0, (prob.nview, 6, 16)).astype(np.float64)
    rbar = np.full_like(y, 0.3)
    u = rng.uniform(0.5, 3, xk.shape)
    beta = 0.7
    s = oracle.sensitivity(prob.mu, psf, prob.dy, ang)
    xn = oracle.em_step_reg(xk, y, rbar, u, beta, prob.mu, psf, prob.dy, ang, s=s)
    ybar = oracle.forward(xk, prob.mu, psf, prob.dy, ang) + rbar
    e = oracle.back(y / ybar, prob.mu, psf, prob.dy, ang)
    d = s - beta * u
    resid = beta * xn ** 2 + d * xn - xk * e
    scale = np.abs(xk * e).max()
    assert np.abs(resid).max() <= 1e-12 * scale
    assert np.all(xn >= 0)
    # and large beta pulls the update towards u
    xb = oracle.em_step_reg(xk, y, rbar, u, 1e9, prob.mu, psf, prob.dy, ang, s=s)
    np.testing.assert_allclose(xb, u, rtol=1e-5)


# ------------------------------------------------------------------ OSEM (ordered subsets of views)
def test_osem_subsets_partition_the_views():
    subs = oracle.osem_subsets(12, 4)
    allv = np.sort(np.concatenate(subs))
    np.testing.assert_array_equal(allv, np.arange(12))
    assert [list(s) for s in subs] == [[0, 4, 8], [1, 5, 9], [2, 6, 10], [3, 7, 11]]


def test_osem_with_one_subset_is_mlem():
    prob, psf, ang = _em_problem()
    rng = np.random.default_rng(41)
    y = rng.poisson(5.0, (prob.nview, 6, 16)).astype(np.float64)
    rbar = np.full_like(y, 0.3)
    x = np.ones((6, 16, 16))
    np.testing.assert_array_equal(oracle.osem_step(x, y, rbar, prob.mu, psf, prob.dy, ang, 1),
                                  oracle.em_step(x, y, rbar, prob.mu, psf, prob.dy, ang))


def test_osem_last_subset_preserves_its_counts():
    # with rbar = 0 each sub-iteration satisfies sum_j (A_S'1)_j x_j = sum_{i in S} y_i
    prob, psf, ang = _em_problem()
    y = np.random.default_rng(42).poisson(5.0, (prob.nview, 6, 16)).astype(np.float64)
    x = oracle.osem_step(np.ones((6, 16, 16)), y, None, prob.mu, psf, prob.dy, ang, 3)
    last = oracle.osem_subsets(prob.nview, 3)[-1]
    s_last = oracle.sensitivity(prob.mu, psf, prob.dy, ang[last])
    assert abs(np.sum(s_last * x) - y[last].sum()) <= 1e-11 * y[last].sum()
    assert np.all(x >= 0)


def test_osem_fixed_point_at_truth():
    prob, psf, ang = _em_problem()
    xt = prob.x.astype(np.float64) + 0.1
    y = oracle.forward(xt, prob.mu, psf, prob.dy, ang)
    np.testing.assert_allclose(oracle.osem_step(xt, y, None, prob.mu, psf, prob.dy, ang, 4), xt, rtol=1e-12)


def test_osem_iteration_advances_further_than_mlem():
    # the reason for subsets: one pass over M subsets makes about M updates' progress
    prob, psf, ang = _em_problem()
    xt = prob.x.astype(np.float64)
    ybar = oracle.forward(xt, prob.mu, psf, prob.dy, ang) * 20
    y = np.random.default_rng(43).poisson(ybar).astype(np.float64)
    x0 = np.full_like(xt, xt.mean())
    ll = lambda x: oracle.poisson_loglik(x, y, None, prob.mu, psf, prob.dy, ang)
    x_em = oracle.em_step(x0, y, None, prob.mu, psf, prob.dy, ang)
    x_os = oracle.osem_step(x0, y, None, prob.mu, psf, prob.dy, ang, 4)
    assert ll(x_os) > ll(x_em) > ll(x0)


# ------------------------------------------------------------------ three-pass rotation (reading R13)
# Section II-A names 3-pass 1D linear interpolation as the alternative image
# rotation.  Pins: the shear product is the rotation matrix (algebra), each
# pass is scipy's order-1 resampling along one axis, quarter turns are the
# lattice permutations, a smooth blob turns by +theta about the centre, mass
# is conserved exactly (each pass shifts rows), the adjoint is the dense
# transpose, and the projector built on it is adjoint and count-preserving.
def _shears(phi):
    """(x, y) = (i - c, j - c) shear matrices Sx(tan(phi/2)), Sy(-sin(phi))."""
    return (np.array([[1.0, np.tan(phi / 2)], [0.0, 1.0]]),
            np.array([[1.0, 0.0], [-np.sin(phi), 1.0]]))


def _scipy_pull(img, m):
    """out(p) = img(m (p - c) + c) by scipy's order-1 resampling, zero outside; m acts on (x, y)."""
    n = img.shape[0]
    c = 0.5 * (n - 1)
    mm = np.array([[m[1, 1], m[1, 0]], [m[0, 1], m[0, 0]]])  # ndimage order: (row j, column i)
    off = np.array([c, c]) - mm @ np.array([c, c])
    return ndimage.affine_transform(img, mm, offset=off, order=1, mode="grid-constant", cval=0.0)


def test_rotation3_shear_product_is_the_rotation():
    for phi in np.linspace(-np.pi / 4, np.pi / 4, 9):
        sx, sy = _shears(phi)
        r = np.array([[np.cos(phi), np.sin(phi)], [-np.sin(phi), np.cos(phi)]])  # R(-phi): output -> source
        np.testing.assert_allclose(sx @ sy @ sx, r, rtol=0, atol=1e-15)


@pytest.mark.parametrize("theta", [0.3, 1.0, 2.2, 3.9, 5.5, -0.6])
def test_rotation3_passes_match_scipy(theta):
    rng = np.random.default_rng(21)
    img = rng.uniform(-1, 1, (13, 13))
    q = int(np.rint(theta / (np.pi / 2)))
    phi = theta - q * np.pi / 2
    sx, sy = _shears(phi)
    ref = _scipy_pull(_scipy_pull(_scipy_pull(np.rot90(img, -(q % 4)), sx), sy), sx)
    np.testing.assert_allclose(oracle.rotate3_slice(img, theta), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("quarter", [0, 1, 2, 3, 4])
def test_rotation3_quarter_turns_are_lattice_permutations(quarter):
    rng = np.random.default_rng(22)
    img = rng.uniform(0, 1, (10, 10))
    got = oracle.rotate3_slice(img, quarter * np.pi / 2)
    np.testing.assert_array_equal(got, np.rot90(img, -quarter))
    np.testing.assert_array_equal(got, oracle.rotate_slice(img, quarter * np.pi / 2))


@pytest.mark.parametrize("theta", [0.4, 1.9, 3.3, 5.0])
def test_rotation3_turns_a_blob_by_theta(theta):
    n, sig = 48, 3.0
    c = 0.5 * (n - 1)
    jj, ii = np.mgrid[0:n, 0:n].astype(np.float64)

    def blob(px, py):
        return np.exp(-((ii - px) ** 2 + (jj - py) ** 2) / (2 * sig * sig))

    p0 = np.array([9.0, -5.0])
    got = oracle.rotate3_slice(blob(*(p0 + c)), theta)
    # content turns by +theta (reading R1): the centre moves to R(theta) p0
    r = np.array([[np.cos(theta), -np.sin(theta)], [np.sin(theta), np.cos(theta)]])
    want = blob(*(r @ p0 + c))
    # three linear passes smooth a sigma = 3 px blob by a few percent of its peak;
    # turning the other way (or about another centre) misses it by ~1
    assert np.abs(got - want).max() < 0.05
    assert np.abs(got - blob(*(r.T @ p0 + c))).max() > 0.5
    # and it agrees with the bilinear rotation to the same accuracy
    assert np.abs(got - oracle.rotate_slice(blob(*(p0 + c)), theta)).max() < 0.05


@pytest.mark.parametrize("theta", [0.35, 2.6, 4.1])
def test_rotation3_conserves_mass_inside_the_circle(theta):
    n = 32
    c = 0.5 * (n - 1)
    jj, ii = np.mgrid[0:n, 0:n]
    rng = np.random.default_rng(23)
    img = rng.uniform(0, 1, (n, n)) * (((ii - c) ** 2 + (jj - c) ** 2) < (0.3 * n) ** 2)
    got = oracle.rotate3_slice(img, theta)
    assert abs(got.sum() - img.sum()) <= 1e-12 * img.sum()
    # bilinear rotation is only approximately mass-preserving
    assert abs(oracle.rotate_slice(img, theta).sum() - img.sum()) > 1e-6 * img.sum()


@pytest.mark.parametrize("theta", [0.4, 2.0, 4.4])
def test_rotation3_adjoint_is_dense_transpose(theta):
    n = 8
    R = np.stack([oracle.rotate3_slice(e.reshape(n, n), theta).ravel() for e in np.eye(n * n)], axis=1)
    Rt = np.stack([oracle.rotate3_adjoint_slice(e.reshape(n, n), theta).ravel() for e in np.eye(n * n)], axis=1)
    np.testing.assert_allclose(Rt, R.T, rtol=0, atol=1e-15)


def test_forward3_quarter_turn_views_equal_bilinear():
    prob = synthetic.random_problem(24, nx=12, nz=4, nview=4, px=3, pz=5, mu_scale=0.2)
    ang = np.arange(4) * np.pi / 2
    a = oracle.forward(prob.x, prob.mu, prob.psf, 1.0, ang, rotation="3pass")
    b = oracle.forward(prob.x, prob.mu, prob.psf, 1.0, ang, rotation="bilinear")
    np.testing.assert_array_equal(a, b)


def test_dense_adjoint3_small():
    prob = synthetic.random_problem(25, nx=8, nz=4, nview=5, px=3, pz=3, symmetric=False, mu_scale=0.3)
    ang = oracle.default_angles(5) + 0.2
    N, M = 8 * 8 * 4, 8 * 4 * 5
    A = np.stack([oracle.forward(e.reshape(4, 8, 8), prob.mu, prob.psf, 1.0, ang, nthreads=1, rotation="3pass").ravel()
                  for e in np.eye(N)], axis=1)
    B = np.stack([oracle.back(e.reshape(5, 4, 8), prob.mu, prob.psf, 1.0, ang, nthreads=1, rotation="3pass").ravel()
                  for e in np.eye(M)], axis=1)
    assert np.linalg.norm(A.T - B) / np.linalg.norm(A) < 1e-14
    # a different operator from the bilinear projector away from quarter turns
    Ab = np.stack([oracle.forward(e.reshape(4, 8, 8), prob.mu, prob.psf, 1.0, ang, nthreads=1).ravel()
                   for e in np.eye(N)], axis=1)
    assert np.linalg.norm(A - Ab) > 1e-3 * np.linalg.norm(A)


def test_em3_preserves_counts_with_zero_background():
    prob, psf, ang = _em_problem()
    rng = np.random.default_rng(26)
    y = rng.poisson(5.0, (prob.nview, 6, 16)).astype(np.float64)
    s = oracle.sensitivity(prob.mu, psf, prob.dy, ang, rotation="3pass")
    x = np.ones((6, 16, 16))
    for _ in range(2):
        x = oracle.em_step(x, y, None, prob.mu, psf, prob.dy, ang, s=s, rotation="3pass")
        assert abs(np.sum(s * x) - y.sum()) <= 1e-11 * y.sum()


# ------------------------------------------------------------------ EM update gradients (Eqs. (7)-(8))
def _central(f, x, h):
    return (f(x + h) - f(x - h)) / (2.0 * h)


@pytest.mark.parametrize("beta", [0.0, 0.05, 0.7, 30.0])
def test_em_root_vjp_matches_finite_differences(beta):
    """The implicit-function derivatives of the update (e/q, x/q, beta x+/q) against
    central differences of em_root itself, element by element, at points where
    d = s - beta u takes both signs (the two closed forms of the root)."""
    rng = np.random.default_rng(31)
    n = 400
    x, e = rng.uniform(0.2, 3.0, n), rng.uniform(0.2, 3.0, n)
    s, u = rng.uniform(0.5, 2.0, n), rng.uniform(0.0, 4.0, n)
    if beta >= 0.5:  # both closed forms of the root are exercised
        d = s - beta * u
        assert (d > 0).any() and (d < 0).any()
    g = rng.normal(0, 1, n)
    gx, ge, gu = oracle.em_root_vjp(x, e, s, u, beta, g)
    h = 1e-6
    for got, var in ((gx, "x"), (ge, "e"), (gu, "u")):
        def f(t):
            args = {"x": x, "e": e, "u": u}
            args[var] = t
            return oracle.em_root(args["x"], args["e"], s, args["u"], beta)
        want = g * _central(f, {"x": x, "e": e, "u": u}[var], h)
        np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-9, err_msg=f"d/d{var}, beta={beta}")
    if beta == 0:
        assert not gu.any()


def test_em_root_vjp_zero_where_the_guard_applies():
    x, e = np.array([1.0, 2.0]), np.array([1.0, 0.0])
    s, u = np.array([0.0, -1.0]), np.zeros(2)
    gx, ge, gu = oracle.em_root_vjp(x, e, s, u, 0.0, np.ones(2))
    assert not gx.any() and not ge.any() and not gu.any()
    # beta > 0, d >= 0 with x e = 0 and d = 0: the root is 0 and so is the gradient
    gx, ge, gu = oracle.em_root_vjp(np.array([0.0]), np.array([0.0]), np.array([1.0]), np.array([1.0]), 1.0,
                                    np.ones(1))
    assert gx[0] == ge[0] == gu[0] == 0


def test_em_ratio_vjp_matches_finite_differences():
    rng = np.random.default_rng(32)
    n = 300
    ybar, y, rbar, g = rng.uniform(0.5, 4, n), rng.poisson(3.0, n).astype(float), rng.uniform(0, 1, n), rng.normal(0, 1, n)
    got = oracle.em_ratio_vjp(ybar, y, rbar, g)
    want = g * _central(lambda t: oracle.em_ratio(t, y, rbar), ybar, 1e-6)
    np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-9)
    # guard: ybar + rbar <= 0 gives ratio 0 and gradient 0
    assert oracle.em_ratio(np.array([-1.0]), np.array([2.0]), np.array([0.5]))[0] == 0
    assert oracle.em_ratio_vjp(np.array([-1.0]), np.array([2.0]), np.array([0.5]), np.ones(1))[0] == 0
