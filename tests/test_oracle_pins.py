"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks retypes an oracle formula: each compares the oracle with
an independent construction (the projection matrix built from a known frame,
3-D ray geometry, closed-form Radon transforms of Gaussians and ellipsoids,
exact chord lengths, affine data that bilinear interpolation reproduces,
adjoint identities between separately written loops, finite differences, and
second-order convergence of the whole chain to the phantom).
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2410_14900_gb300 import synth


def _desc(w: synth.Workload):
    return w.desc_dict()


def _small_circle(V=16, H=24, W=32, p=2.0, n_mu=36, n_s=32, N=(8, 10, 12), ds=None):
    o = synth.circle_orbit(V)
    ds = p if ds is None else ds
    vox = p * synth.SID_MM / synth.SDD_MM
    d = dict(n_views=V, det_rows=H, det_cols=W, n_mu=n_mu, n_s=n_s, pitch=p, ds=ds,
             vol_x=N[2], vol_y=N[1], vol_z=N[0], voxel=(vox, vox, vox),
             vol_center=(0.0, 0.0, 0.0), closed_orbit=1)
    P = synth.projection_matrices(o, H, W, p)
    return o, d, P


# --------------------------------------------------------------- geometry
@pytest.mark.parametrize("kind", ["circle", "sinusoid", "circle_arc", "tilted"])
def test_geometry_recovers_frame_from_matrix(kind):
    """Source, detector frame, D and principal point come back from P (Fig. 1)."""
    o = {"circle": lambda: synth.circle_orbit(12),
         "sinusoid": lambda: synth.sinusoid_orbit(12),
         "circle_arc": lambda: synth.circle_arc_orbit(8, 5),
         "tilted": lambda: synth.tilted_sinusoid_orbit(12)}[kind]()
    H, W, p = 30, 40, 0.8
    P = synth.projection_matrices(o, H, W, p)
    scale = np.linspace(-3.0, 2.0, o.n_views)[:, None, None]  # any nonzero scale
    scale[scale == 0] = 1.0
    d = dict(n_views=o.n_views, pitch=p, det_rows=H, det_cols=W, closed_orbit=1,
             vol_center=(0.0, 0.0, 0.0))
    geom = orc.Geometry(d, P * scale, o.vdl)
    for i in range(o.n_views):
        np.testing.assert_allclose(geom.source(i), o.sources[i], rtol=0, atol=1e-9)
        lx, ly, lz = geom.frame(i)
        np.testing.assert_allclose(lx, o.lx[i], atol=1e-12)
        np.testing.assert_allclose(ly, o.ly[i], atol=1e-12)
        np.testing.assert_allclose(lz, o.lz[i], atol=1e-12)
        assert abs(geom.D(i) - o.sdd) < 1e-9
        cu, cv = geom.principal_point(i)
        assert abs(cu - (W - 1) / 2) < 1e-9 and abs(cv - (H - 1) / 2) < 1e-9


def test_geometry_rejects_bad_matrices():
    o = synth.circle_orbit(4)
    P = synth.projection_matrices(o, 8, 8, 1.0)
    d = dict(n_views=4, pitch=1.0, det_rows=8, det_cols=8, closed_orbit=1)
    bad = P.copy()
    bad[1, 0, :3] *= 1.5            # non-square pixels
    with pytest.raises(ValueError):
        orc.Geometry(d, bad)
    bad = P.copy()
    bad[2, 2, :3] = 0.0             # no depth row
    with pytest.raises(ValueError):
        orc.Geometry(d, bad)


def test_tangent_finite_difference_matches_analytic():
    """a'(lambda) dlambda by central differences converges to the analytic tangent."""
    for V in (90, 180):
        o = synth.sinusoid_orbit(V)
        P = synth.projection_matrices(o, 8, 8, 1.0)
        d = dict(n_views=V, pitch=1.0, det_rows=8, det_cols=8, closed_orbit=1)
        geom = orc.Geometry(d, P, None)
        err = max(np.linalg.norm(geom.tangent(i) - o.vdl[i]) for i in range(V))
        scale = np.linalg.norm(o.vdl[0])
        assert err < 2e-3 * scale * (90 / V) ** 2 * 1.01 + 1e-12
    # open orbit: one-sided ends
    o = synth.circle_arc_orbit(10, 6)
    P = synth.projection_matrices(o, 8, 8, 1.0)
    d = dict(n_views=o.n_views, pitch=1.0, det_rows=8, det_cols=8, closed_orbit=0)
    geom = orc.Geometry(d, P, None)
    np.testing.assert_allclose(geom.tangent(0), o.sources[1] - o.sources[0], atol=1e-12)
    np.testing.assert_allclose(geom.tangent(o.n_views - 1),
                               o.sources[-1] - o.sources[-2], atol=1e-12)


# --------------------------------------------------------- pointwise weights
def test_cosine_weight_is_ray_cosine():
    """w_cos = cos(angle between the pixel ray and the principal ray) (Eq. 6/7)."""
    o, d, P = _small_circle()
    geom = orc.Geometry(d, P, o.vdl)
    for i in (0, 5):
        rays = synth.pixel_rays(o, i, d["det_rows"], d["det_cols"], d["pitch"])
        cosang = rays @ (-o.lz[i])
        w = orc.cosine_weight(geom, i, np.ones((d["det_rows"], d["det_cols"])))
        np.testing.assert_allclose(w, cosang, rtol=1e-13)


def test_detector_weight_is_squared_ray_length():
    """w_d = |pixel - source|^2 (Eq. 11)."""
    o, d, P = _small_circle()
    geom = orc.Geometry(d, P, o.vdl)
    H, W, p = d["det_rows"], d["det_cols"], d["pitch"]
    i = 3
    O = o.sources[i] - o.sdd * o.lz[i]
    x = (np.arange(W) - (W - 1) / 2) * p
    y = (np.arange(H) - (H - 1) / 2) * p
    pts = O + x[None, :, None] * o.lx[i] + y[:, None, None] * o.ly[i]
    l2 = np.sum((pts - o.sources[i]) ** 2, -1)
    np.testing.assert_allclose(orc.detector_weight(geom, i, np.ones((H, W))), l2, rtol=1e-13)


def test_redundancy_K_circle_closed_form():
    """Circle: |a'.theta| = R D |cos mu| / sqrt(s^2+D^2) per radian (Eq. 14, R*D reading)."""
    V = 24
    o, d, P = _small_circle(V=V)
    geom = orc.Geometry(d, P, o.vdl)
    n_mu, n_s, ds, D, R = d["n_mu"], d["n_s"], d["ds"], o.sdd, synth.SID_MM
    mu = np.arange(n_mu) * math.pi / n_mu
    sh = (np.arange(n_s) - (n_s - 1) / 2 + 0.5) * ds
    dphi = 2 * math.pi / V
    ref = -(R * D * np.abs(np.cos(mu))[:, None] * dphi / np.sqrt(sh ** 2 + D ** 2)[None, :]
            ) / (4 * math.pi ** 2 * np.sqrt(sh ** 2 + D ** 2)[None, :])
    ref[:, -1] = 0.0
    for i in (0, 7, 19):
        np.testing.assert_allclose(orc.redundancy_K(geom, i), ref, rtol=1e-12,
                                   atol=1e-14 * np.abs(ref).max())


def test_redundancy_K_uses_plane_normal():
    """|v.theta| with theta the normal of the plane through the source and the line."""
    o = synth.circle_arc_orbit(6, 4)
    H, W, p, n_mu, n_s = 16, 20, 1.5, 12, 20
    P = synth.projection_matrices(o, H, W, p)
    d = dict(n_views=o.n_views, det_rows=H, det_cols=W, n_mu=n_mu, n_s=n_s, pitch=p, ds=p,
             closed_orbit=0)
    geom = orc.Geometry(d, P, o.vdl)
    i = 8  # an arc view
    K = orc.redundancy_K(geom, i)
    O = o.sources[i] - o.sdd * o.lz[i]
    for m in (0, 3, 7):
        mu = m * math.pi / n_mu
        for k in (0, 9, 17):
            s = (k - (n_s - 1) / 2 + 0.5) * p
            # two points of the detector line x cos mu + y sin mu = s
            e_u = math.cos(mu) * o.lx[i] + math.sin(mu) * o.ly[i]
            e_v = -math.sin(mu) * o.lx[i] + math.cos(mu) * o.ly[i]
            p1, p2 = O + s * e_u, O + s * e_u + 10.0 * e_v
            th = np.cross(p1 - o.sources[i], p2 - o.sources[i])
            th /= np.linalg.norm(th)
            ref = -abs(o.vdl[i] @ th) / (4 * math.pi ** 2 * math.hypot(s, o.sdd))
            tol = 1e-13 * np.linalg.norm(o.vdl[i]) / (4 * math.pi ** 2 * o.sdd)
            assert abs(K[m, k] - ref) <= 1e-12 * abs(ref) + tol


# ----------------------------------------------------------------- A2d
def test_radon_axis_angles_are_column_and_row_sums():
    rng = np.random.default_rng(3)
    H, W, p = 12, 16, 0.7
    img = rng.normal(size=(H, W))
    n_mu = 4  # mu = 0, pi/4, pi/2, 3pi/4
    R = orc.radon(img, p, n_mu, W, p)  # s grid aligned with columns
    np.testing.assert_allclose(R[0], p * img.sum(0), rtol=1e-13)
    Rv = orc.radon(img, p, n_mu, H, p)  # s grid aligned with rows (H even)
    np.testing.assert_allclose(Rv[2], p * img.sum(1), rtol=1e-12, atol=1e-12)


def test_radon_constant_image_chord_length():
    """Interior lines through a constant image measure the chord of the row band."""
    H, W, p = 20, 300, 1.0
    R = orc.radon(np.ones((H, W)), p, 64, 64, p)
    for m in range(64):
        mu = m * math.pi / 64
        if not (4 * m <= 64 or 4 * m >= 192):
            continue
        # every line with |s| small crosses all rows well inside the columns
        np.testing.assert_allclose(R[m, 24:40], H * p / abs(math.cos(mu)), rtol=1e-12)


def test_radon_gaussian_closed_form():
    """A2d of exp(-r^2/2 sigma^2) is sqrt(2 pi) sigma exp(-s^2/2 sigma^2)."""
    errs = []
    for n in (64, 128):
        p = 64.0 / n
        sig = 5.0
        x = (np.arange(n) - (n - 1) / 2) * p
        X, Y = np.meshgrid(x, x)
        img = np.exp(-(X ** 2 + Y ** 2) / (2 * sig ** 2))
        R = orc.radon(img, p, 30, n, p)
        s = (np.arange(n) - (n - 1) / 2) * p
        ref = math.sqrt(2 * math.pi) * sig * np.exp(-s ** 2 / (2 * sig ** 2))
        errs.append(np.abs(R - ref[None]).max() / ref.max())
    assert errs[1] < 2e-3
    assert errs[0] / errs[1] > 3.0  # O(p^2)


def test_radon_transpose_dense():
    """The scatter loop is the exact transpose of the gather loop (dense matrices)."""
    H, W, p, n_mu, n_s, ds = 5, 6, 1.0, 7, 8, 1.0
    A = np.zeros((n_mu * n_s, H * W))
    for c in range(H * W):
        e = np.zeros(H * W)
        e[c] = 1.0
        A[:, c] = orc.radon(e.reshape(H, W), p, n_mu, n_s, ds).ravel()
    AT = np.zeros((H * W, n_mu * n_s))
    for c in range(n_mu * n_s):
        e = np.zeros(n_mu * n_s)
        e[c] = 1.0
        AT[:, c] = orc.radon_T(e.reshape(n_mu, n_s), H, W, p, ds).ravel()
    np.testing.assert_allclose(AT, A.T, rtol=0, atol=1e-15)
    assert np.count_nonzero(A) > 0


def test_radon_adjoint_identity_off_centre():
    rng = np.random.default_rng(0)
    H, W, p, n_mu, n_s, ds = 17, 23, 0.9, 31, 29, 1.1
    x = rng.normal(size=(H, W))
    y = rng.normal(size=(n_mu, n_s))
    lhs = np.sum(orc.radon(x, p, n_mu, n_s, ds, cu=9.3, cv=7.1) * y)
    rhs = np.sum(x * orc.radon_T(y, H, W, p, ds, cu=9.3, cv=7.1))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# ------------------------------------------------------------ derivatives
def test_derivatives_exact_on_polynomials_and_adjoint():
    ds = 0.5
    k = np.arange(12.0)
    s = (k - 5.5) * ds
    R = np.tile(3 * s ** 2 - s + 2, (2, 1))
    Df = orc.deriv_f(R, ds)
    sh = s + ds / 2
    np.testing.assert_allclose(Df[:, :-1], np.tile(6 * sh - 1, (2, 1))[:, :-1], rtol=1e-12)
    assert np.all(Df[:, -1] == 0)
    DbDf = orc.deriv_b(Df, ds)
    np.testing.assert_allclose(DbDf[:, 1:-1], 6.0, rtol=1e-12)  # second derivative
    rng = np.random.default_rng(1)
    for f, fT in ((orc.deriv_f, orc.deriv_f_T), (orc.deriv_b, orc.deriv_b_T)):
        x = rng.normal(size=(3, 12))
        y = rng.normal(size=(3, 12))
        assert abs(np.sum(f(x, ds) * y) - np.sum(x * fT(y, ds))) < 1e-12


# -------------------------------------------------------------- Grangeat
def _plane_normal(o, i, mu, s):
    O = o.sources[i] - o.sdd * o.lz[i]
    e_u = math.cos(mu) * o.lx[i] + math.sin(mu) * o.ly[i]
    e_v = -math.sin(mu) * o.lx[i] + math.cos(mu) * o.ly[i]
    p1 = O + s * e_u
    p2 = p1 + e_v
    th = np.cross(p2 - o.sources[i], p1 - o.sources[i])
    th /= np.linalg.norm(th)
    # orientation: +e_u side (the half space the s axis points into)
    if th @ e_u < 0:
        th = -th
    return th


def _dRf_gauss(b, th, rho):
    """d/drho of the 3-D Radon transform of a Gaussian blob (closed form)."""
    n = np.diag(b.axes) @ b.rot.T @ th
    h = np.linalg.norm(n)
    t = rho - b.center @ th
    detA = np.prod(b.axes)
    return -2 * math.pi * b.rho * detA * t / h ** 3 * math.exp(-t * t / (2 * h * h))


def _grangeat_error(o, i, n, p):
    H = W = n
    n_mu, n_s, ds = 24, n, p
    P = synth.projection_matrices(o, H, W, p)
    d = dict(n_views=o.n_views, det_rows=H, det_cols=W, n_mu=n_mu, n_s=n_s, pitch=p, ds=ds,
             closed_orbit=1)
    geom = orc.Geometry(d, P, o.vdl)
    b = synth.Blob("gauss", np.array([2.0, -1.5, 2.5]), np.array([3.0, 4.0, 3.5]),
                   synth.random_rotation(np.random.default_rng(5)), 0.8)
    g = synth.project_phantom([b], o, H, W, p)
    # the blob's shadow lies inside the detector (no truncated line integrals)
    edge = max(np.abs(g[i][[0, -1], :]).max(), np.abs(g[i][:, [0, -1]]).max())
    assert edge < 1e-6 * g[i].max()
    S = orc.grangeat(geom, i, g[i])
    ref = np.zeros_like(S)
    for m in range(n_mu):
        mu = m * math.pi / n_mu
        for k in range(n_s - 1):
            s = (k - (n_s - 1) / 2 + 0.5) * ds
            th = _plane_normal(o, i, mu, s)
            ref[m, k] = _dRf_gauss(b, th, o.sources[i] @ th)
    err = np.abs(S - ref).max() / np.abs(ref).max()
    big = np.abs(ref) > 0.3 * np.abs(ref).max()
    return err, np.all(np.sign(S[big]) == np.sign(ref[big]))


@pytest.mark.parametrize("orbit", ["circle", "arc"])
def test_grangeat_relation_gaussian(orbit):
    """S(mu, s, lambda) = d/drho Rf(theta, a.theta)  (Eq. 1 -> Eq. 6/7).

    Joseph's interpolation error changes from one s-bin to the next at oblique
    angles, so after the s-difference the error falls at first order in p.
    """
    if orbit == "circle":
        o, i = synth.circle_orbit(8), 3
    else:
        o, i = synth.circle_arc_orbit(4, 5), 6
    e1, sign1 = _grangeat_error(o, i, 80, 1.0)
    e2, sign2 = _grangeat_error(o, i, 160, 0.5)
    assert sign1 and sign2          # the sign is part of the relation
    assert e2 < 1.2e-2, (e1, e2)
    assert e1 / e2 > 1.7, (e1, e2)


def test_grangeat_relation_ellipsoid_integral():
    """For an ellipsoid, sum_k S * ds over s reproduces the jump of Rf (=0) and
    int S ds between two s values equals the difference of the closed-form Rf
    along the plane family (Grangeat, discrete s-integral)."""
    o = synth.circle_orbit(8)
    i = 1
    H = W = 200
    p = 0.4
    n_mu, n_s, ds = 12, 200, 0.4
    P = synth.projection_matrices(o, H, W, p)
    d = dict(n_views=8, det_rows=H, det_cols=W, n_mu=n_mu, n_s=n_s, pitch=p, ds=ds,
             closed_orbit=1)
    geom = orc.Geometry(d, P, o.vdl)
    b = synth.Blob("ellipsoid", np.array([3.0, 2.0, -4.0]), np.array([10.0, 8.0, 12.0]),
                   synth.random_rotation(np.random.default_rng(2)), 1.0)
    g = synth.project_phantom([b], o, H, W, p)
    S = orc.grangeat(geom, i, g[i])
    # S is the rho-derivative in the plane family rotating about the detector
    # line; the total over s of S*ds(rho)/ds vanishes because Rf returns to 0.
    for m in range(n_mu):
        mu = m * math.pi / n_mu
        sh = (np.arange(n_s) - (n_s - 1) / 2 + 0.5) * ds
        rho = np.array([o.sources[i] @ _plane_normal(o, i, mu, s) for s in sh])
        drho = np.gradient(rho)
        total = np.sum(S[m, :-1] * drho[:-1])
        assert abs(total) < 1e-2 * np.abs(S[m] * drho).sum()


# --------------------------------------------------------------- filter
def test_filter_adjoint_identity_and_weight_gradient():
    o, d, P = _small_circle(V=5, H=10, W=12, n_mu=9, n_s=12)
    d["closed_orbit"] = 1
    geom = orc.Geometry(d, P, o.vdl)
    rng = np.random.default_rng(4)
    B = 2
    g = rng.normal(size=(B, 5, 10, 12))
    Wr = rng.uniform(0.2, 0.8, size=(5, 9, 12))
    G = rng.normal(size=g.shape)
    gF = orc.filter(geom, g, Wr)
    gg, gW = orc.filter_adjoint(geom, g, G, Wr)
    # linear in g
    x = rng.normal(size=g.shape)
    lhs = np.sum(orc.filter(geom, x, Wr) * G)
    _, _ = orc.filter_adjoint(geom, x, G, Wr, want_grad_W=False)
    gx, _ = orc.filter_adjoint(geom, g, G, Wr, want_grad_W=False)
    assert abs(lhs - np.sum(x * gx)) < 1e-10 * abs(lhs)
    # linear in W: directional derivative equals <grad_W, dW>
    dW = rng.normal(size=Wr.shape)
    dW[:, :, -1] = 0.0
    lhs = np.sum((orc.filter(geom, g, Wr + dW) - gF) * G)
    assert abs(lhs - np.sum(gW * dW)) < 1e-10 * abs(lhs)
    assert np.all(gW[:, :, -1] == 0)


# --------------------------------------------------------- backprojection
def test_backprojection_affine_data_closed_form():
    """Bilinear interpolation reproduces affine detector data exactly, so
    f(X) = sum_i (alpha u_i(X) + beta v_i(X) + gamma) / |X - a_i|^2 (Eq. 5)."""
    o, d, P = _small_circle(V=7, H=40, W=48, N=(6, 7, 5))
    geom = orc.Geometry(d, P, o.vdl)
    H, W = d["det_rows"], d["det_cols"]
    al, be, ga = 0.3, -0.2, 1.7
    jj, rr = np.meshgrid(np.arange(W), np.arange(H))
    gF = np.broadcast_to(al * jj + be * rr + ga, (7, H, W)).copy()
    f = orc.backproject(geom, gF)[0]
    xs, ys, zs = synth.voxel_centers((6, 7, 5), d["voxel"])
    ref = np.zeros_like(f)
    for i in range(7):
        for iz, z in enumerate(zs):
            for iy, y in enumerate(ys):
                for ix, x in enumerate(xs):
                    X = np.array([x, y, z, 1.0])
                    U, Vv, w = P[i] @ X
                    u, v = U / w, Vv / w
                    assert 0 < u < W - 1 and 0 < v < H - 1
                    ref[iz, iy, ix] += (al * u + be * v + ga) / np.sum((X[:3] - o.sources[i]) ** 2)
    np.testing.assert_allclose(f, ref, rtol=1e-12)


def test_backprojection_adjoint_points_relu_and_depth():
    o, d, P = _small_circle(V=4, H=9, W=11, N=(5, 6, 7))
    geom = orc.Geometry(d, P, o.vdl)
    rng = np.random.default_rng(7)
    gF = rng.normal(size=(2, 4, 9, 11))
    vol = orc.backproject(geom, gF)
    gv = rng.normal(size=vol.shape)
    gg = orc.backproject_adjoint(geom, gv)
    assert abs(np.sum(vol * gv) - np.sum(gF * gg)) < 1e-11 * np.abs(vol * gv).sum()
    flat = np.array([0, 17, 100, 5 * 6 * 7 - 1])
    pts = orc.backproject_points(geom, gF[1], flat)
    np.testing.assert_allclose(pts, vol[1].ravel()[flat], rtol=1e-14)
    r = orc.backproject(geom, gF, relu=True)
    np.testing.assert_array_equal(r, np.maximum(vol, 0))
    acc = orc.backproject(geom, gF, vol=vol)
    np.testing.assert_allclose(acc, 2 * vol, rtol=1e-14)
    # a volume around the source: voxels behind it (depth <= 0) get nothing
    d2 = dict(d, n_views=1, vol_x=3, vol_y=3, vol_z=1, voxel=(800.0, 800.0, 1.0))
    g2 = orc.Geometry(d2, P[:1], o.vdl[:1])
    out = orc.backproject(g2, np.ones((1, 1, 9, 11)))[0, 0]
    # the column x = +800 lies beyond the source at (750,0,0): behind it.  Its
    # centre voxel would land on the principal point if depth were ignored.
    assert np.all(out[:, 2] == 0.0)
    assert out[1, 1] > 0.0


# ------------------------------------------------------------ full chain
def _chain_error(V, n, p, n_mu, N=48, ds=None):
    o = synth.circle_orbit(V)
    vox = 80.0 / N
    ds = p if ds is None else ds
    n_s = int(round(n * p / ds))
    d = dict(n_views=V, det_rows=n, det_cols=n, n_mu=n_mu, n_s=n_s, pitch=p, ds=ds,
             vol_x=N, vol_y=N, vol_z=1, voxel=(vox, vox, vox), closed_orbit=1)
    P = synth.projection_matrices(o, n, n, p)
    geom = orc.Geometry(d, P, o.vdl)
    blobs = [synth.Blob("gauss", np.array([0.0, 0.0, 0.0]), np.array([6.0, 6.0, 6.0]),
                        np.eye(3), 1.0),
             synth.Blob("gauss", np.array([12.0, -5.0, 0.0]), np.array([3.0, 5.0, 4.0]),
                        synth.random_rotation(np.random.default_rng(9)), 0.7)]
    g = synth.project_phantom(blobs, o, n, n, p)
    f = orc.reconstruct(geom, g[None])[0, 0]
    gt = synth.phantom_volume(blobs, (1, N, N), (vox, vox, vox))[0]
    c = (np.arange(N) - (N - 1) / 2) * vox
    roi = np.hypot(*np.meshgrid(c, c)) < 35.0  # inside the field of view (40 mm)
    return np.linalg.norm((f - gt)[roi]) / np.linalg.norm(gt[roi]), f[roi].sum() / gt[roi].sum()


def test_full_chain_converges_to_phantom_on_circle_midplane():
    """Eq. 12 with the analytic circle weights (Eq. 14, M = 1/2) reconstructs the
    midplane of a smooth phantom; the error falls at second order with the
    detector pitch, and the mean is right (sign and -1/4pi^2 normalisation)."""
    e1, m1 = _chain_error(64, 64, 2.0, 180)
    e2, m2 = _chain_error(128, 128, 1.0, 360)
    assert e2 < 0.015, (e1, e2)
    assert e1 / e2 > 3.0, (e1, e2)
    assert abs(m1 - 1.0) < 0.03 and abs(m2 - 1.0) < 0.01, (m1, m2)
    # s-bins coarser than the pixels: the A2d^T normalisation ds/p^2 matters
    e3, m3 = _chain_error(128, 128, 1.0, 360, ds=1.25)
    assert e3 < 0.02 and abs(m3 - 1.0) < 0.01, (e3, m3)


def test_mse_gradient_matches_central_differences():
    """dL/dW and dL/dg by reverse mode equal FP64 central differences (L quadratic)."""
    o, d, P = _small_circle(V=4, H=8, W=10, n_mu=6, n_s=10, N=(3, 4, 5))
    geom = orc.Geometry(d, P, o.vdl)
    rng = np.random.default_rng(11)
    g = rng.normal(size=(1, 4, 8, 10))
    Wr = np.full((4, 6, 10), 0.5)
    tgt = rng.normal(size=(1, 3, 4, 5))

    def loss(g_, W_):
        r = orc.backproject(geom, orc.filter(geom, g_, W_)) - tgt
        return 0.5 * np.sum(r * r)

    r = orc.backproject(geom, orc.filter(geom, g, Wr)) - tgt
    gg, gW = orc.filter_adjoint(geom, g, orc.backproject_adjoint(geom, r), Wr)
    h = 1e-3
    for (v, m, k) in [(0, 1, 2), (2, 4, 5), (3, 0, 7)]:
        e = np.zeros_like(Wr)
        e[v, m, k] = h
        fd = (loss(g, Wr + e) - loss(g, Wr - e)) / (2 * h)
        assert abs(fd - gW[v, m, k]) <= 1e-8 * max(1.0, abs(fd))
    for idx in [(0, 0, 3, 4), (0, 2, 5, 1)]:
        e = np.zeros_like(g)
        e[idx] = h
        fd = (loss(g + e, Wr) - loss(g - e, Wr)) / (2 * h)
        assert abs(fd - gg[idx]) <= 1e-8 * max(1.0, abs(fd))


# ------------------------------------------------------ Crofton weights (Eq. 9)
def test_crofton_weights_are_one_half_on_a_circle():
    """Every plane through a circle point meets the circle once more, with the
    same |a'.theta| by symmetry: M = 1/2 (Eq. 14).  Planes tangent to the
    orbit at the source (K ~ 0) carry no weight and are excluded."""
    o, d, P = _small_circle(V=48, H=40, W=40, p=3.0, n_mu=24, n_s=40)
    geom = orc.Geometry(d, P, o.vdl)
    M = orc.crofton_weights(geom, m=2)[:, :, :-1]
    K = np.stack([orc.redundancy_K(geom, i) for i in range(d["n_views"])])[:, :, :-1]
    use = np.abs(K) > 0.01 * np.abs(K).max()
    assert use.mean() > 0.9
    # the crossing's tangent is interpolated linearly between views
    assert np.abs(M[use] - 0.5).max() < 5e-3


def _arc_crossings(o, i, th, n_circle):
    """Independent count of the plane's intersections with a circle+arc orbit
    (the circle in z = 0, the arc in the x-z plane), excluding view i."""
    ai = o.sources[i]
    R = np.linalg.norm(o.sources[0])
    c = th @ ai
    rxy = math.hypot(th[0], th[1])
    n_circ = 0
    if rxy > 0:
        dist = abs(c) / rxy
        if abs(dist - R) < 1e-3 * R:
            return None           # near tangency: count not robust
        n_circ = 2 if dist < R else 0
    psi = np.linspace(-math.pi / 6, math.pi / 6, 20001)
    f = (R * np.cos(psi)) * th[0] + (R * np.sin(psi)) * th[2] - c
    psi_i = math.atan2(ai[2], ai[0])
    sgn = np.sign(f)
    idx = np.nonzero(sgn[:-1] * sgn[1:] < 0)[0]
    roots = psi[idx]
    # drop the root at the source itself; reject roots near the arc ends
    roots = roots[np.abs(roots - psi_i) > 2e-3]
    if np.any(np.abs(np.abs(roots) - math.pi / 6) < 0.05):
        return None
    if i < n_circle:
        # source on the circle: the circle's second crossing, arc crossings
        return (n_circ - 1 if n_circ else 0) + len(roots)
    return n_circ + len(roots)


def test_crofton_m0_is_the_crofton_symbol_on_circle_plus_arc():
    """m = 0, no taper: M = 1/n with n the number of intersections of the plane
    with the orbit (Eq. 3's Crofton symbol), counted independently."""
    nc, na = 60, 21
    o = synth.circle_arc_orbit(nc, na)
    H = W = 48
    p = 2.5
    P = synth.projection_matrices(o, H, W, p)
    d = dict(n_views=o.n_views, det_rows=H, det_cols=W, n_mu=16, n_s=48, pitch=p, ds=p,
             closed_orbit=0)
    geom = orc.Geometry(d, P, o.vdl)
    M = orc.crofton_weights(geom, [(0, True), (nc, False)], m=0, taper=0)
    checked = 0
    for i in (3, 25, nc + 4, nc + 10, nc + 17):
        lx, ly, lz = o.lx[i], o.ly[i], o.lz[i]
        for m_ in range(16):
            mu = m_ * math.pi / 16
            for k in range(0, 47, 3):
                s = (k - 23.5 + 0.5) * p
                th = (o.sdd * math.cos(mu) * lx + o.sdd * math.sin(mu) * ly + s * lz)
                th = th / np.linalg.norm(th)
                if abs(o.vdl[i] @ th) < 1e-3 * np.linalg.norm(o.vdl[i]):
                    continue
                n_other = _arc_crossings(o, i, th, nc)
                if n_other is None:
                    continue
                assert abs(M[i, m_, k] - 1.0 / (1 + n_other)) < 1e-12, (i, m_, k, n_other)
                checked += 1
    assert checked > 200


def test_crofton_weights_reconstruct_circle_plus_arc_off_midplane():
    """A circle plus arc satisfies Tuy's condition: with the Eq. 9 weights the
    reconstruction of blobs away from the circle's plane is accurate, where
    the circle's weight 1/2 leaves large cone-beam errors."""
    nc, na, n, p, nmu, N = 72, 30, 72, 1.6, 90, 30
    o = synth.circle_arc_orbit(nc, na)
    vox = 60.0 / N
    d = dict(n_views=o.n_views, det_rows=n, det_cols=n, n_mu=nmu, n_s=n, pitch=p, ds=p,
             vol_x=N, vol_y=N, vol_z=N, voxel=(vox, vox, vox), closed_orbit=0)
    geom = orc.Geometry(d, synth.projection_matrices(o, n, n, p), o.vdl)
    blobs = [synth.Blob("gauss", np.array([0.0, 0.0, 14.0]), np.array([5.0, 5.0, 5.0]),
                        np.eye(3), 1.0),
             synth.Blob("gauss", np.array([8.0, -6.0, -10.0]), np.array([3.0, 4.0, 3.5]),
                        np.eye(3), 0.6)]
    g = synth.project_phantom(blobs, o, n, n, p)
    gt = synth.phantom_volume(blobs, (N, N, N), (vox, vox, vox))
    c = (np.arange(N) - (N - 1) / 2) * vox
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    roi = (X ** 2 + Y ** 2 + Z ** 2) < 26 ** 2
    M = orc.crofton_weights(geom, [(0, True), (nc, False)], m=2, taper=3)
    err = {}
    for name, Wt in (("half", None), ("crofton", M)):
        f = orc.reconstruct(geom, g[None], Wt)[0]
        err[name] = np.linalg.norm((f - gt)[roi]) / np.linalg.norm(gt[roi])
    assert err["crofton"] < 0.04, err
    assert err["half"] > 4 * err["crofton"], err


# ------------------------------------------------ Gaussian smoothing of W
def test_gauss_smooth_is_scipys_mirror_filter():
    """Separable 121-tap Gaussian (sigma 20) with mirror ends: the same as
    scipy's gaussian_filter1d(mode='mirror', truncate=3) along mu and s."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(21)
    W = rng.normal(size=(3, 150, 97))
    got = orc.gauss_smooth(W, 20.0, 60)
    ref = W.copy()
    v = ndimage.gaussian_filter1d(W[:, :, :-1], 20.0, axis=1, mode="mirror", truncate=3.0)
    ref[:, :, :-1] = ndimage.gaussian_filter1d(v, 20.0, axis=2, mode="mirror", truncate=3.0)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(W).max())
    np.testing.assert_array_equal(got[:, :, -1], W[:, :, -1])  # unused entry passes


def test_gauss_smooth_closed_forms_and_adjoint():
    # constants are kept (unit-sum taps); a delta far from the ends spreads
    # into the sampled Gaussian profile; short lines mirror repeatedly
    W = np.full((2, 40, 33), 0.7)
    np.testing.assert_allclose(orc.gauss_smooth(W, 20.0, 60), W, atol=1e-14)
    D = np.zeros((1, 301, 302))
    D[0, 150, 150] = 1.0
    S = orc.gauss_smooth(D, 5.0, 15)
    t = np.arange(-15, 16)
    g = np.exp(-0.5 * t ** 2 / 25.0)
    g /= g.sum()
    np.testing.assert_allclose(S[0, 135:166, 135:166], np.outer(g, g), atol=1e-15)
    assert abs(S.sum() - 1.0) < 1e-12
    rng = np.random.default_rng(22)
    x = rng.normal(size=(2, 37, 29))
    y = rng.normal(size=(2, 37, 29))
    lhs = np.sum(orc.gauss_smooth(x, 20.0, 60) * y)
    rhs = np.sum(x * orc.gauss_smooth(y, 20.0, 60, adjoint=True))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
