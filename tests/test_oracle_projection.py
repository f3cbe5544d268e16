"""Pins of the oracle's projection pieces against mathematics the paper fixes.

Sec. 3.2 (equidistant model r_d = f theta, x_p / y_p equations), Sec. 4.2 (J_phi),
Sec. 4.3 (dJ/d{x_c, y_c, z_c} with S1..S8), Sec. 3.1 (Sigma_p = J W Sigma W^T J^T).
Each test checks the oracle against something other than its own formula: an invariant of
the model, a limit, central finite differences, or an arbitrary-precision derivative.
"""
import math

import numpy as np
import pytest

import oracle

mpmath = pytest.importorskip("mpmath")


def _rand_points(rng, n, zmin=-3.0):
    pts = []
    while len(pts) < n:
        p = rng.normal(size=3) * 2.0
        p[2] = rng.uniform(zmin, 4.0)
        th = math.atan2(math.hypot(p[0], p[1]), p[2])
        if np.linalg.norm(p) > 0.3 and th < math.pi - 0.1:
            pts.append(p)
    return np.array(pts)


def test_equidistance_invariant():
    """r_d = f * theta with theta the angle between mu_c and the optical axis (Sec. 3.2),
    and the image point lies on the ray of (x_c, y_c) from the principal point."""
    rng = np.random.default_rng(10)
    f, cx, cy = 457.3, 320.5, 240.25
    for p in _rand_points(rng, 200):
        xy = oracle.project_point(p, f, f, cx, cy)
        mp = [mpmath.mpf(float(v)) for v in p]
        theta = mpmath.acos(mp[2] / mpmath.sqrt(mp[0] ** 2 + mp[1] ** 2 + mp[2] ** 2))
        r = math.hypot(xy[0] - cx, xy[1] - cy)
        assert abs(r - f * float(theta)) <= 1e-9 * max(1.0, r)
        # same direction as (x_c, y_c)
        lz = math.hypot(p[0], p[1])
        assert abs((xy[0] - cx) * p[1] - (xy[1] - cy) * p[0]) <= 1e-9 * r * lz
        assert (xy[0] - cx) * p[0] + (xy[1] - cy) * p[1] >= 0


def test_on_axis_maps_to_principal_point():
    for z in (0.25, 1.0, 7.5):
        xy = oracle.project_point([0.0, 0.0, z], 300.0, 250.0, 128.0, 96.0)
        assert xy[0] == 128.0 and xy[1] == 96.0


def test_small_angle_limit_is_pinhole():
    """theta -> 0: the equidistant image tends to the pinhole image c + f (x/z, y/z); the gap
    is f (t - atan t) ~ f t^3 / 3 (t = l_z / z)."""
    f = 500.0
    for t in (1e-6, 1e-4, 1e-3, 1e-2, 5e-2):
        for ang in (0.3, 2.0, 4.1):
            z = 2.0
            x, y = t * z * math.cos(ang), t * z * math.sin(ang)
            xy = oracle.project_point([x, y, z], f, f, 0.0, 0.0)
            pin = np.array([f * x / z, f * y / z])
            gap = np.linalg.norm(xy - pin)
            assert abs(gap - f * (t - math.atan(t))) <= 1e-9 * f * t + 1e-12


def _phi_mp(p, fx, fy):
    x, y, z = p
    lz = mpmath.sqrt(x * x + y * y)
    th = mpmath.atan2(lz, z)
    return fx * th * x / lz, fy * th * y / lz


def _jac_mp(p, fx, fy):
    """Exact J by 50-digit numerical differentiation of phi."""
    mpmath.mp.dps = 50
    P = [mpmath.mpf(float(v)) for v in p]
    J = np.zeros((2, 3))
    for r in range(2):
        for c in range(3):
            def fr(s, r=r, c=c):
                Q = list(P)
                Q[c] = Q[c] + s
                return _phi_mp(Q, fx, fy)[r]
            J[r, c] = float(mpmath.diff(fr, 0))
    return J


@pytest.mark.parametrize("t", [1e-8, 1e-5, 3e-3, 9.9e-3, 1.01e-2, 0.1, 0.7, None])
def test_jacobian_vs_arbitrary_precision(t):
    """J_phi of Sec. 4.2 (with f on the theta terms) equals the exact derivative, including
    the near-axis series region and z_c < 0."""
    rng = np.random.default_rng(11)
    fx, fy = 500.0, 400.0
    pts = _rand_points(rng, 6) if t is None else [
        np.array([t * 1.7 * math.cos(a), t * 1.7 * math.sin(a), 1.7]) for a in (0.4, 2.5)]
    for p in pts:
        J = oracle.jacobian(p, fx, fy)
        Jx = _jac_mp(p, fx, fy)
        assert np.allclose(J, Jx, rtol=1e-11, atol=1e-11 * np.abs(Jx).max())


def test_jacobian_finite_differences():
    rng = np.random.default_rng(12)
    fx, fy = 610.0, 590.0
    for p in _rand_points(rng, 100):
        J = oracle.jacobian(p, fx, fy)
        h = 1e-6 * max(1.0, np.linalg.norm(p))
        Jfd = np.zeros((2, 3))
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            Jfd[:, c] = (oracle.project_point(p + e, fx, fy) - oracle.project_point(p - e, fx, fy)) / (2 * h)
        assert np.allclose(J, Jfd, rtol=1e-7, atol=1e-7 * np.abs(J).max())


def test_printed_jacobian_lacks_focal_length():
    """The matrix printed in Sec. 4.2 omits f on its theta terms: at (0.3, -0.7, 1.1),
    f = (500, 400) its [0,0] entry is 48.35 while the derivative is 383.56."""
    x, y, z = 0.3, -0.7, 1.1
    fx, fy = 500.0, 400.0
    lz2, l2 = x * x + y * y, x * x + y * y + z * z
    lz = math.sqrt(lz2)
    th = math.atan2(lz, z)
    printed00 = fx * x * x * z / (lz2 * l2) + y * y * th / lz ** 3
    J = oracle.jacobian([x, y, z], fx, fy)
    assert abs(printed00 - 48.35) < 0.01
    assert abs(J[0, 0] - 383.56) < 0.01
    assert abs(J[0, 0] - _jac_mp([x, y, z], fx, fy)[0, 0]) < 1e-9


def _dJ_fd(p, fx, fy):
    out = []
    h = 1e-5 * max(1.0, np.linalg.norm(p))
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        out.append((oracle.jacobian(p + e, fx, fy) - oracle.jacobian(p - e, fx, fy)) / (2 * h))
    return out


def test_jacobian_grad_finite_differences():
    """dJ/dx_c, dJ/dy_c, dJ/dz_c (Sec. 4.3, S1..S8) against central differences of J."""
    rng = np.random.default_rng(13)
    fx, fy = 500.0, 420.0
    for p in _rand_points(rng, 80):
        dJ = oracle.jacobian_grad(p, fx, fy)
        fd = _dJ_fd(p, fx, fy)
        scale = max(np.abs(d).max() for d in fd)
        for a, b in zip(dJ, fd):
            assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * scale)


@pytest.mark.parametrize("t", [1e-7, 1e-4, 5e-3, 9.99e-3, 1.001e-2, 3e-2])
def test_jacobian_grad_near_axis_arbitrary_precision(t):
    """Near the axis S7, S8 cancel to order t^4; the oracle's series must match the exact
    second derivatives of phi (50 digits)."""
    mpmath.mp.dps = 60
    fx, fy = 480.0, 510.0
    for a in (0.7, 3.9):
        p = np.array([t * 2.3 * math.cos(a), t * 2.3 * math.sin(a), 2.3])
        dJ = oracle.jacobian_grad(p, fx, fy)
        P = [mpmath.mpf(float(v)) for v in p]
        for k in range(3):
            ex = np.zeros((2, 3))
            for r in range(2):
                for c in range(3):
                    def fr(s1, s2, r=r, c=c):
                        Q = list(P)
                        Q[c] += s1
                        Q[k] += s2
                        return _phi_mp(Q, fx, fy)[r]
                    ex[r, c] = float(mpmath.diff(fr, (0, 0), (1, 1)))
            sc = np.abs(ex).max()
            assert np.allclose(dJ[k], ex, rtol=1e-9, atol=1e-9 * sc), (k, dJ[k], ex)


def test_printed_dJdy_entry_has_wrong_focal_length():
    """Sec. 4.3 prints dJ/dy_c[0,2] = 2 f_y x y / l2^2; the derivative is 2 f_x x y / l2^2.
    The two differ by f_y / f_x whenever f_x != f_y."""
    p = np.array([0.4, -0.3, 1.2])
    fx, fy = 500.0, 400.0
    dJ = oracle.jacobian_grad(p, fx, fy)
    fd = _dJ_fd(p, fx, fy)
    l2 = float(p @ p)
    printed = 2 * fy * p[0] * p[1] / l2 ** 2
    assert abs(dJ[1][0, 2] - fd[1][0, 2]) < 1e-6 * abs(fd[1][0, 2])
    assert abs(printed / fd[1][0, 2] - fy / fx) < 1e-6


def _scene1(mu, s, q=(1.0, 0.0, 0.0, 0.0), opac=0.8, dc=0.3):
    return dict(means=np.array([mu], np.float64), scales=np.array([s], np.float64),
                quats=np.array([q], np.float64), opacities=np.array([opac], np.float64),
                sh=np.full((1, 1, 3), dc), sh_degree=0)


def test_isotropic_on_axis_covariance_closed_form():
    """Isotropic Gaussian of scale s on the optical axis at distance z: J = (f/z)[I | 0]
    there, so Sigma_p = ((f s / z)^2 + 0.3) I exactly (Sec. 3.1 / 4.3 + the dilation)."""
    f, s, z = 300.0, 0.05, 2.0
    for W, centre in [(np.eye(3), np.zeros(3)),
                      (np.array([[0.0, -1, 0], [1, 0, 0], [0, 0, 1]]), np.zeros(3))]:
        mu = W.T @ np.array([0.0, 0.0, z])
        cam = dict(W=W, b=-W @ centre, fx=f, fy=f, cx=64.0, cy=64.0, width=128, height=128)
        G = oracle.project(_scene1(mu, [s, s, s], q=(0.3, 0.1, -0.5, 0.8)), cam)[0]
        a, b, c = G[oracle.F["cov"]:oracle.F["cov"] + 3]
        want = (f * s / z) ** 2 + 0.3
        assert abs(a - want) < 1e-12 * want and abs(c - want) < 1e-12 * want and abs(b) < 1e-12


def test_covariance_psd_and_det_bound():
    from paper_2409_04751_gb300 import scenes
    scene, cams = scenes.config0()
    G = oracle.project(scene, cams[0])
    vis = G[:, 0] > 0
    a, b, c = (G[vis, oracle.F["cov"] + k] for k in range(3))
    det = a * c - b * b
    assert np.all(a >= 0.3) and np.all(c >= 0.3) and np.all(det >= 0.09 - 1e-12)
    sig = G[vis, oracle.F["sig"]:oracle.F["sig"] + 6]
    for row in sig[:200]:
        S = np.array([[row[0], row[1], row[2]], [row[1], row[3], row[4]], [row[2], row[4], row[5]]])
        assert np.linalg.eigvalsh(S).min() > -1e-15


def _real_sh_scipy(l, m, d):
    """Real SH with the Condon-Shortley phase, built from scipy's complex Y_l^m."""
    from scipy.special import sph_harm_y
    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0])
    if m == 0:
        return sph_harm_y(l, 0, theta, phi).real
    Y = sph_harm_y(l, abs(m), theta, phi)  # includes (-1)^m
    return math.sqrt(2.0) * (Y.real if m > 0 else Y.imag)


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(14)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y, _ = oracle.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                assert abs(Y[l * l + l + m] - _real_sh_scipy(l, m, d)) < 1e-12


def test_sh_basis_orthonormal():
    """Gauss-Legendre x uniform-phi quadrature of Y_i Y_j over the sphere is the identity."""
    xs, ws = np.polynomial.legendre.leggauss(12)
    phis = np.linspace(0, 2 * math.pi, 24, endpoint=False)
    gram = np.zeros((16, 16))
    for x, w in zip(xs, ws):
        st = math.sqrt(1 - x * x)
        for ph in phis:
            d = np.array([st * math.cos(ph), st * math.sin(ph), x])
            Y, _ = oracle.sh_basis(3, d)
            gram += w * (2 * math.pi / len(phis)) * np.outer(Y, Y)
    assert np.allclose(gram, np.eye(16), atol=1e-12)


def test_sh_gradient_tangent_fd():
    rng = np.random.default_rng(15)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        _, dY = oracle.sh_basis(3, d)
        v = rng.normal(size=3)
        v -= d * (d @ v)
        v /= np.linalg.norm(v)
        h = 1e-6
        dp = (d + h * v) / np.linalg.norm(d + h * v)
        dm = (d - h * v) / np.linalg.norm(d - h * v)
        fd = (oracle.sh_basis(3, dp)[0] - oracle.sh_basis(3, dm)[0]) / (2 * h)
        assert np.allclose(dY @ v, fd, atol=1e-8)
