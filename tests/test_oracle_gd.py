"""Pins of the oracle's Galerkin-Difference (and Catmull-Rom) interpolant.

Paper: Sec. II-B (Eq. 10-13) and Appendix A (p = 3 basis and the central
difference weights of D^(1,3)); Eq. 7 for Catmull-Rom.  Each check ties the
oracle to something other than itself: the defining conditions of the basis
solved exactly, the printed coefficients (tests/golden), polynomial
reproduction, continuity, and the measured convergence order.
"""
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_2506_18579_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        key, rest = parts[0], parts[1:]
        if rest and rest[0] in ("xi", "xi+1", "xi+2", "xi-1", "-"):  # shift label column
            rest = rest[1:]
        rows[key] = [Fr(x) for x in rest]
    return rows


def _solve_exact(A, b):
    """Gauss-Jordan elimination over the rationals."""
    n = len(A)
    M = [list(A[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [x / piv for x in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[i][n] for i in range(n)]


def _weights_from_conditions():
    """Per-node weight polynomials w_a(t), a = -1..2, of the degree-5 cell
    interpolant defined by Appendix A: it takes the nodal values at t = -1, 0,
    1, 2 and, at t = 0 and t = 1, the slope h D^(1,3) u = -u_{j-1}/2 + u_{j+1}/2.
    Returns {a: [c0..c5]} (coefficients of t^0..t^5), exact rationals."""
    eta = {-1: Fr(-1, 2), 0: Fr(0), 1: Fr(1, 2)}
    out = {}
    for a in (-1, 0, 1, 2):
        u = {n: Fr(1 if n == a else 0) for n in (-1, 0, 1, 2, 3)}
        rows, rhs = [], []
        for t in (-1, 0, 1, 2):  # value conditions
            rows.append([Fr(t) ** k for k in range(6)])
            rhs.append(u[t])
        for t in (0, 1):  # slope conditions from the central-difference operator
            rows.append([k * Fr(t) ** (k - 1) if k > 0 else Fr(0) for k in range(6)])
            rhs.append(sum(eta[o] * u.get(t + o, Fr(0)) for o in (-1, 0, 1)))
        out[a] = _solve_exact(rows, rhs)
    return out


def _expand_shifted(coeffs_desc):
    """Coefficients (t^0..t^5) of sum c_k s^k with s = t (the cell-local argument)."""
    c = list(reversed(coeffs_desc))  # c0..c5
    return c + [Fr(0)] * (6 - len(c))


def test_appendix_basis_follows_from_its_conditions():
    """The printed pieces (golden) are exactly the unique solution of the
    Appendix A conditions: w_{-1} = psi_1, w_0 = psi_0, w_1 = psi_{-1},
    w_2 = psi_{-2}, each in its own shifted argument."""
    g = _read_golden("gd_p3_appendix.txt")
    assert g["eta"] == [Fr(-1, 2), Fr(0), Fr(1, 2)]
    derived = _weights_from_conditions()
    pairs = {-1: "psi_1", 0: "psi_0", 1: "psi_m1", 2: "psi_m2"}
    for a, name in pairs.items():
        assert _expand_shifted(g[name]) == derived[a], name
    # partition of unity, exactly
    assert [sum(derived[a][k] for a in derived) for k in range(6)] == [1, 0, 0, 0, 0, 0]


def test_oracle_psi_matches_derived_basis(orc):
    derived = _weights_from_conditions()
    for t in np.linspace(0.0, 1.0, 37)[:-1]:
        for a in (-1, 0, 1, 2):
            c = [float(x) for x in derived[a]]
            exp_v = sum(c[k] * t ** k for k in range(6))
            exp_d = sum(k * c[k] * t ** (k - 1) for k in range(1, 6))
            v, d = orc.gd_psi(t - a)
            assert v == pytest.approx(exp_v, abs=1e-14)
            assert d == pytest.approx(exp_d, abs=1e-13)


def test_psi_node_values_support_symmetry(orc):
    assert orc.gd_psi(0.0)[0] == 1.0
    for x in (-2.0, -1.0, 1.0, 2.0, -2.5, 2.5, 7.0):
        assert abs(orc.gd_psi(x)[0]) < 1e-15
    for x in np.linspace(0.01, 1.99, 23):
        assert orc.gd_psi(x)[0] == pytest.approx(orc.gd_psi(-x)[0], abs=1e-14)
        assert orc.gd_psi(x)[1] == pytest.approx(-orc.gd_psi(-x)[1], abs=1e-13)


def test_psi_is_c1_but_not_c2(orc):
    eps = 1e-7
    jumps2 = []
    for x in (-2.0, -1.0, 0.0, 1.0, 2.0):
        vl, dl = orc.gd_psi(x - eps)
        vr, dr = orc.gd_psi(x + eps)
        assert vl == pytest.approx(vr, abs=1e-6)
        assert dl == pytest.approx(dr, abs=1e-5)
        d2l = (orc.gd_psi(x - eps)[1] - orc.gd_psi(x - 1e-3)[1]) / (1e-3 - eps)
        d2r = (orc.gd_psi(x + 1e-3)[1] - orc.gd_psi(x + eps)[1]) / (1e-3 - eps)
        jumps2.append(abs(d2l - d2r))
    assert max(jumps2) > 0.1  # second derivative jumps at the nodes


def _alt_only_grid(values, dalt=1.0, alt0=0.0, b0=0.0):
    n = len(values)
    spec = wl.GridSpec(n_lat=4, n_lon=4, n_alt=n, lat0_deg=0.0, lon0_deg=0.0, alt0_km=alt0,
                       dlat_deg=1.0, dlon_deg=1.0, dalt_km=dalt, b0_tesla=b0)
    ne = np.broadcast_to(np.asarray(values, float), spec.shape).copy()
    return spec, ne


def test_node_slope_is_central_difference(orc):
    rng = np.random.default_rng(3)
    u = rng.normal(size=12)
    spec, ne = _alt_only_grid(u, dalt=2.5)
    g = orc.Grid(spec, ne)
    for j in range(1, 11):
        out = orc.ne(g, 1.5, 1.5, j * 2.5)
        assert out[0] == pytest.approx(u[j], abs=1e-13)
        assert out[3] == pytest.approx((u[j + 1] - u[j - 1]) / (2 * 2.5), abs=1e-12)


def test_1d_reproduces_quadratics_not_cubics(orc):
    x = np.arange(10.0)
    for deg, exact in ((0, True), (1, True), (2, True), (3, False)):
        spec, ne = _alt_only_grid(x ** deg)
        g = orc.Grid(spec, ne)
        errs = []
        for t in np.linspace(0.0, 9.0, 91):  # includes the first/last cells (ghost nodes)
            out = orc.ne(g, 1.0, 1.0, t)
            errs.append(abs(out[0] - t ** deg))
            errs.append(abs(out[3] - deg * t ** (deg - 1) if deg else out[3]))
        if exact:
            assert max(errs) < 1e-10, deg
        else:
            assert max(errs) > 1e-3


def test_brute_force_cell_polynomial(orc):
    """On an interior cell the interpolant equals the degree-5 polynomial
    solved from 4 values + 2 central-difference slopes (numpy, floating)."""
    rng = np.random.default_rng(7)
    u = rng.normal(size=8)
    spec, ne = _alt_only_grid(u)
    g = orc.Grid(spec, ne)
    for j in range(1, 6):
        A = np.array([[float(t) ** k for k in range(6)] for t in (-1, 0, 1, 2)] +
                     [[k * float(t) ** (k - 1) if k else 0.0 for k in range(6)] for t in (0, 1)])
        b = np.array([u[j - 1], u[j], u[j + 1], u[j + 2],
                      (u[j + 1] - u[j - 1]) / 2, (u[j + 2] - u[j]) / 2])
        c = np.linalg.solve(A, b)
        for t in np.linspace(0, 1, 11)[:-1]:
            out = orc.ne(g, 1.0, 1.0, j + t)
            assert out[0] == pytest.approx(np.polyval(c[::-1], t), abs=1e-12)


def test_3d_tensor_quadratic_exact_including_faces(orc):
    rng = np.random.default_rng(11)
    spec = wl.GridSpec(n_lat=6, n_lon=7, n_alt=8, lat0_deg=10.0, lon0_deg=100.0, alt0_km=60.0,
                       dlat_deg=2.0, dlon_deg=1.5, dalt_km=10.0)
    C = rng.normal(size=(3, 3, 3))
    lat, lon, alt = spec.axes()

    def q(la, lo, al):
        a, b, c = (la - 15) / 10, (lo - 104) / 9, (al - 95) / 70
        pa, pb, pc = np.array([1, a, a * a]), np.array([1, b, b * b]), np.array([1, c, c * c])
        v = np.einsum("ijk,i,j,k->", C, pa, pb, pc)
        da = np.einsum("ijk,i,j,k->", C, np.array([0, 1, 2 * a]), pb, pc) / 10
        db = np.einsum("ijk,i,j,k->", C, pa, np.array([0, 1, 2 * b]), pc) / 9
        dc = np.einsum("ijk,i,j,k->", C, pa, pb, np.array([0, 1, 2 * c])) / 70
        return v, da, db, dc

    ne = np.array([[[q(a, b, c)[0] for c in alt] for b in lon] for a in lat])
    g = orc.Grid(spec, ne)
    pts = rng.uniform([lat[0], lon[0], alt[0]], [lat[-1], lon[-1], alt[-1]], size=(60, 3))
    pts[:4] = [[lat[0], lon[0], alt[0]], [lat[-1], lon[-1], alt[-1]],
               [lat[0] + 0.3, lon[-1] - 0.2, alt[0] + 1], [lat[-1], lon[0], alt[-1] - 0.5]]
    for p in pts:
        out = orc.ne(g, *p)
        v, da, db, dc = q(*p)
        assert out[4] == 1.0
        np.testing.assert_allclose(out[:4], [v, da, db, dc], rtol=1e-10, atol=1e-10)


def test_outside_box_is_free_space(orc):
    spec, ne = _alt_only_grid(np.ones(6) * 5.0, alt0=60.0, dalt=10.0)
    g = orc.Grid(spec, ne)
    for p in ((1.0, 1.0, 59.0), (1.0, 1.0, 111.0), (-0.5, 1.0, 80.0), (1.0, 3.5, 80.0)):
        out = orc.ne(g, *p)
        assert out[4] == 0.0 and np.all(out[:4] == 0.0)
    assert orc.ne(g, 1.0, 1.0, 60.0)[0] == pytest.approx(5.0)


def test_convergence_order_on_chapman(orc):
    """Value error O(h^3), gradient error O(h^2): the printed p = 3 basis
    reproduces quadratics, so neither the O(h^p) of Eq. 18 nor the O(h^{p+1})
    quoted in Sec. IV-A holds for it; the measured orders are asserted."""
    hm, H = 300.0, 60.0
    f = lambda z: np.exp(0.5 * (1 - (z - hm) / H - np.exp(-(z - hm) / H)))
    df = lambda z: f(z) * 0.5 * (-1 / H + np.exp(-(z - hm) / H) / H)
    zs = np.linspace(150.0, 450.0, 301)
    ev, eg = [], []
    hs = (16.0, 8.0, 4.0, 2.0)
    for h in hs:
        n = int(round(600 / h)) + 1
        spec, ne = _alt_only_grid(f(np.arange(n) * h), dalt=h)
        g = orc.Grid(spec, ne)
        out = np.array([orc.ne(g, 1.0, 1.0, z) for z in zs])
        ev.append(np.max(np.abs(out[:, 0] - f(zs))))
        eg.append(np.max(np.abs(out[:, 3] - df(zs))))
    ov = np.log2(np.array(ev[:-1]) / np.array(ev[1:]))
    og = np.log2(np.array(eg[:-1]) / np.array(eg[1:]))
    assert np.all(ov[1:] > 2.7), ov
    assert np.all(og[1:] > 1.8), og


def test_catmull_rom_matches_eq7_and_reproduces_quadratics(orc):
    g = _read_golden("catmull_rom_eq7.txt")
    for t in np.linspace(0, 1, 17):
        w = orc.cr_weights(t)
        for a, name in zip(range(4), ("w_m1", "w_0", "w_1", "w_2")):
            c = [float(x) for x in g[name]]  # t^3..t^0
            assert w[a] == pytest.approx(np.polyval(c, t), abs=1e-14)
    x = np.arange(10.0)
    spec, ne = _alt_only_grid(x ** 2)
    gr = orc.Grid(spec, ne, interp="cr")
    for t in np.linspace(1.0, 8.0, 29):
        out = orc.ne(gr, 1.0, 1.0, t)
        assert out[0] == pytest.approx(t * t, abs=1e-10)
