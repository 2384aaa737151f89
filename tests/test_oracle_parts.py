"""Pins for the FP64 oracle's parts, each against something other than the
oracle itself: closed forms the paper states, invariants, a library routine
for a special case, or brute force on tiny inputs."""
import json
import math
import os

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as ss

from paper_2608_23245_b300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _rad_cell(c):
    return (c[0], c[1], c[2], math.radians(c[3]), math.radians(c[4]), math.radians(c[5]))


def _metric(cell):
    """Real-space metric tensor from the six cell constants (textbook form,
    independent of the orthogonalisation convention)."""
    a, b, c, al, be, ga = cell
    return np.array([[a * a, a * b * math.cos(ga), a * c * math.cos(be)],
                     [a * b * math.cos(ga), b * b, b * c * math.cos(al)],
                     [a * c * math.cos(be), b * c * math.cos(al), c * c]])


# ----------------------------------------------------------------- basis ---

@pytest.mark.parametrize("name", [k for k in GOLD["cells"] if not k.startswith("_")])
def test_basis_paper_cells(orc, name):
    """Eq. recip_basis: a*_i . a_j = delta_ij; the real basis reproduces the
    cell's lengths and angles; c || z and b in the yz-plane (Sect. Unit cell
    and reciprocal-space frame); a along x for an orthogonal cell."""
    cell = _rad_cell(GOLD["cells"][name])
    A, As = orc.basis(cell)
    assert np.allclose(As @ A.T, np.eye(3), atol=1e-14)
    assert np.allclose(A @ A.T, _metric(cell), rtol=1e-13, atol=1e-12)
    assert abs(A[2, 0]) < 1e-15 and abs(A[2, 1]) < 1e-15 and A[2, 2] > 0
    assert abs(A[1, 0]) < 1e-15
    if all(abs(x - 90.0) < 1e-12 for x in GOLD["cells"][name][3:]):
        assert abs(A[0, 1]) < 1e-12 and abs(A[0, 2]) < 1e-12


def test_basis_random_triclinic(orc):
    rng = np.random.default_rng(7)
    for _ in range(20):
        ang = np.radians(rng.uniform(70, 115, size=3))
        cell = (*rng.uniform(4, 40, size=3), *ang)
        A, As = orc.basis(cell)
        assert np.allclose(As @ A.T, np.eye(3), atol=1e-13)
        assert np.allclose(A @ A.T, _metric(cell), rtol=1e-12, atol=1e-10)


# ----------------------------------------------------------- reflections ---

def _brute_reflections(cell, dmin, dmax=0.0):
    """Brute force over a generous box with 1/d^2 = h G^-1 h (metric tensor)."""
    Gs = np.linalg.inv(_metric(cell))
    H = [int(math.ceil(1.5 * cell[i] / dmin)) + 1 for i in range(3)]
    out = []
    for h in range(-H[0], H[0] + 1):
        for k in range(-H[1], H[1] + 1):
            for l in range(-H[2], H[2] + 1):
                if h == 0 and k == 0 and l == 0:
                    continue
                v = np.array([h, k, l], dtype=float)
                s2 = v @ Gs @ v
                if s2 <= (1 + 1e-12) / dmin ** 2 and (dmax <= 0 or s2 >= (1 - 1e-12) / dmax ** 2):
                    out.append((h, k, l))
    return np.array(out, dtype=np.int32).reshape(-1, 3)


@pytest.mark.parametrize("cell,dmin,dmax", [
    ((9.0, 9.0, 15.0, math.pi / 2, math.pi / 2, math.pi / 2), 2.5, 0.0),
    ((20.0, 20.0, 28.0, math.pi / 2, math.pi / 2, math.radians(120.0)), 3.0, 0.0),
    (_rad_cell(GOLD["cells"]["cellulose_I_alpha"]), 2.2, 6.0),
    (_rad_cell(GOLD["cells"]["CTA"]), 2.0, 0.0),
])
def test_reflections_brute_force(orc, cell, dmin, dmax):
    """Sect. Structure factors and reflection list: every (h,k,l) != 0 with
    d_min <= d <= d_max, lexicographic; checked against a brute-force scan of
    a larger box using the metric tensor instead of the Cartesian basis."""
    got = orc.reflections(cell, dmin, dmax)
    ref = _brute_reflections(cell, dmin, dmax)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)
    # Friedel mates present, (000) absent, lexicographic order
    s = set(map(tuple, got.tolist()))
    assert all((-h, -k, -l) in s for (h, k, l) in s)
    assert (0, 0, 0) not in s
    keys = got[:, 0].astype(np.int64) * 10 ** 6 + got[:, 1] * 10 ** 3 + got[:, 2]
    assert np.all(np.diff(keys) > 0)


def test_reflection_counts_configs(orc):
    """Whole-sphere counts of the three single-model workloads (reading R1)."""
    for f, n in ((W.config0, 304), (W.config1, 5062)):
        p = f()
        assert len(orc.reflections(p.cell, p.d_min, p.d_max)) == n
    p = W.config0()
    ref = _brute_reflections(p.cell, p.d_min)
    assert len(ref) == 304


# ------------------------------------------------------ structure factors ---

def _one_atom(frac, B=0.0, ff=None, occ=1.0):
    if ff is None:
        ff = np.array([[0, 0, 0, 0, 1, 1, 1, 1, 2.5]], dtype=float)
    return W.Atoms(frac=np.array(frac, dtype=float).reshape(-1, 3), B=np.atleast_1d(np.array(B, dtype=float)),
                   occ=np.atleast_1d(np.array(occ, dtype=float)), elem=np.zeros(len(np.atleast_2d(frac)), np.uint8),
                   ff=np.asarray(ff, dtype=float))


CELL_T = _rad_cell(GOLD["cells"]["cellulose_I_alpha"])


def _s2(cell, hkl):
    Gs = np.linalg.inv(_metric(cell))
    h = np.asarray(hkl, dtype=float)
    return np.einsum("ni,ij,nj->n", h, Gs, h)


def test_sf_single_atom_origin(orc):
    """Eq. structure_factor, one atom at the origin: every phase is 1, so
    F = f(s) exp(-B s^2/4) (real); with a constant form factor c and B = 0,
    F = c exactly; B enters as exp(-B s^2/4) with s = 1/d."""
    hkl = orc.reflections(CELL_T, 2.5)
    F = orc.structure_factors(CELL_T, _one_atom([0, 0, 0]), hkl)
    assert np.allclose(F, 2.5, rtol=0, atol=1e-14)
    B = 17.0
    FB = orc.structure_factors(CELL_T, _one_atom([0, 0, 0], B=B), hkl)
    assert np.allclose(FB.real, 2.5 * np.exp(-B * _s2(CELL_T, hkl) / 4.0), rtol=1e-13)
    assert np.allclose(FB.imag, 0.0, atol=1e-15)


def test_sf_form_factor_limits(orc):
    """f(s) -> sum a_i + c at s -> 0, and -> c for s -> infinity (each
    Gaussian term decays)."""
    ff = np.array([[1.0, 2.0, 0.5, 0.25, 3.0, 10.0, 20.0, 30.0, 0.75]])
    at = _one_atom([0, 0, 0], ff=ff)
    big = (4000.0, 4000.0, 4000.0, math.pi / 2, math.pi / 2, math.pi / 2)
    F = orc.structure_factors(big, at, np.array([[1, 0, 0]], np.int32))
    assert abs(F[0].real - 4.5) < 1e-6
    tiny = (0.05, 0.05, 0.05, math.pi / 2, math.pi / 2, math.pi / 2)
    F = orc.structure_factors(tiny, at, np.array([[1, 1, 1]], np.int32))
    assert abs(F[0].real - 0.75) < 1e-12


def test_sf_phase_and_friedel(orc):
    """A shifted atom multiplies F by exp(2 pi i h.x); Friedel's law
    F(-h) = conj F(h); a lattice translation leaves F unchanged."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, size=3)
    hkl = orc.reflections(CELL_T, 2.0)
    F = orc.structure_factors(CELL_T, _one_atom(x), hkl)
    ref = 2.5 * np.exp(2j * np.pi * (hkl @ x))
    assert np.allclose(F, ref, rtol=0, atol=1e-13)
    p = W.small_triclinic()
    F = orc.structure_factors(p.cell, p.atoms, hkl)
    Fm = orc.structure_factors(p.cell, p.atoms, -hkl)
    assert np.allclose(Fm, np.conj(F), rtol=0, atol=1e-12 * np.abs(F).max())
    shifted = W.Atoms(frac=p.atoms.frac + np.array([1.0, -2.0, 3.0]), B=p.atoms.B, occ=p.atoms.occ,
                      elem=p.atoms.elem, ff=p.atoms.ff)
    Fs = orc.structure_factors(p.cell, shifted, hkl)
    assert np.allclose(Fs, F, rtol=0, atol=1e-11 * np.abs(F).max())


def test_sf_centrosymmetric_and_pair(orc):
    """Atoms in +-x pairs give a real F; two atoms give
    |F|^2 = f1^2 + f2^2 + 2 f1 f2 cos(2 pi h.(x1 - x2))."""
    rng = np.random.default_rng(5)
    xs = rng.uniform(0, 1, size=(10, 3))
    ff = np.array([[1.2, 0.7, 0.3, 0.1, 2.0, 8.0, 15.0, 30.0, 0.4]])
    atoms = W.Atoms(frac=np.concatenate([xs, -xs]), B=np.full(20, 12.0), occ=np.ones(20),
                    elem=np.zeros(20, np.uint8), ff=ff)
    hkl = orc.reflections(CELL_T, 2.0)
    F = orc.structure_factors(CELL_T, atoms, hkl)
    assert np.max(np.abs(F.imag)) < 1e-12 * np.max(np.abs(F))
    ff2 = np.array([[0, 0, 0, 0, 1, 1, 1, 1, 1.3], [0, 0, 0, 0, 1, 1, 1, 1, 0.6]])
    pair = W.Atoms(frac=xs[:2].copy(), B=np.zeros(2), occ=np.ones(2), elem=np.array([0, 1], np.uint8), ff=ff2)
    F = orc.structure_factors(CELL_T, pair, hkl)
    ref = 1.3 ** 2 + 0.6 ** 2 + 2 * 1.3 * 0.6 * np.cos(2 * np.pi * hkl @ (xs[0] - xs[1]))
    assert np.allclose(np.abs(F) ** 2, ref, rtol=1e-12)


# ------------------------------------------------- disorder and lineshapes --

def test_hosemann_scalars_paper_forms(orc):
    """Eq. Ah, Eq. breadth, Eq. Neff and Eq. Ipara in the paper's printed
    form, against the oracle's tanh/sech rewrite."""
    p = W.small_triclinic()
    hkl = orc.reflections(p.cell, p.d_min)
    beta, P, DW = orc.refl_scalars(p, hkl)
    A, _ = orc.basis(p.cell)
    alen = np.linalg.norm(A, axis=1)
    Ah = np.exp(-2 * np.pi ** 2 * np.array(p.br.g)[None, :] ** 2 * hkl.astype(float) ** 2)
    breadth = (1 - Ah) / (1 + Ah)
    Nbase = np.array(p.br.L)[None, :] / alen[None, :]
    ref_beta = np.minimum(1.0, 1.0 / Nbase + breadth)
    assert np.allclose(beta, ref_beta, rtol=1e-13)
    ref_P = np.prod(2 * Ah / (1 + Ah ** 2), axis=1)
    assert np.allclose(P, ref_P, rtol=1e-13)
    # axis damping D(S) = exp(-1/4 sum B_i (S . a^_i)^2), S = D_hkl
    _, As = orc.basis(p.cell)
    D = hkl @ As
    ahat = A / alen[:, None]
    ref_DW = np.exp(-0.25 * np.sum(np.array(p.br.B_axis)[None, :] * (D @ ahat.T) ** 2, axis=1))
    assert np.allclose(DW, ref_DW, rtol=1e-13)


def test_paracrystal_width_h2(orc):
    """Eq. paracrystal_width: for small g the extra breadth grows as
    pi^2 g^2 h^2 (order-squared signature)."""
    p = W.small_lorentz()
    g = 0.002
    hkl = np.array([[h, 0, 0] for h in range(1, 8)], np.int32)
    beta, _, _ = orc.refl_scalars(p, hkl, g=(g, g, g), L=(1e12, 1e12, 1e12))
    h = np.arange(1, 8)
    assert np.allclose(beta[:, 0], np.pi ** 2 * g ** 2 * h ** 2, rtol=1e-3)


@pytest.mark.parametrize("beta", [0.02, 0.1, 0.37, 0.9])
def test_hosemann_lineshape(orc, beta):
    """Eq. Z: K = (1 - phi^2)/(1 - 2 phi cos(2 pi t) + phi^2) with
    phi = (1 - beta)/(1 + beta); equals its Fourier series
    sum_n phi^|n| exp(2 pi i n t); peak 1/beta = (1 + A)/(1 - A); unit
    integral over one period (Eq. breadth)."""
    phi = (1 - beta) / (1 + beta)
    for t in np.linspace(-0.5, 0.5, 41):
        K = orc.lineshape(1, t, beta)
        eqZ = (1 - phi ** 2) / (1 - 2 * phi * math.cos(2 * math.pi * t) + phi ** 2)
        n = np.arange(1, 4000)
        series = 1 + 2 * np.sum(phi ** n * np.cos(2 * np.pi * n * t))
        assert K == pytest.approx(eqZ, rel=1e-12)
        assert K == pytest.approx(series, rel=1e-9)
    assert orc.lineshape(1, 0.0, beta) == pytest.approx((1 + phi) / (1 - phi), rel=1e-13)
    val, _ = si.quad(lambda t: orc.lineshape(1, t, beta), -0.5, 0.5, epsabs=1e-13, epsrel=1e-13, limit=400,
                     points=[0.0])
    assert val == pytest.approx(1.0, rel=1e-9)


@pytest.mark.parametrize("N", [5, 11, 15])
def test_sinc_lineshape_laue(orc, N):
    """Eq. I_shape with integer N: K(0) = N, zeros at t = m/N, and
    K(t) (pi t)^2 / sin^2(pi t) = |sum_{n<N} exp(2 pi i n t)|^2 / N (Eq. laue1d,
    brute-force sum); the non-periodic envelope integrates to 1."""
    beta = 1.0 / N
    assert orc.lineshape(0, 0.0, beta) == pytest.approx(N, rel=1e-14)
    for m in (1, 2, 3):
        assert abs(orc.lineshape(0, m / N, beta)) < 1e-12
    for t in np.linspace(0.003, 0.45, 25):
        lsum = abs(np.sum(np.exp(2j * np.pi * np.arange(N) * t))) ** 2
        K = orc.lineshape(0, t, beta)
        assert K * (math.pi * t) ** 2 / math.sin(math.pi * t) ** 2 == pytest.approx(lsum / N, rel=1e-10)
    val, _ = si.quad(lambda t: orc.lineshape(0, t, beta), -60.0 / N, 60.0 / N, limit=2000, epsabs=1e-12)
    tail = 1.0 / (math.pi ** 2 * 60.0)  # both tails |N t| > 60 of sin^2(pi x)/(pi x)^2, sin^2 averaged to 1/2
    assert val == pytest.approx(1.0 - tail, abs=2e-5)
    assert orc.support(0, beta, 3.0) == pytest.approx(min(3.0 / N, 0.5))


@pytest.mark.parametrize("beta", [0.03, 0.1, 0.3])
def test_gauss_lineshape_matched_breadth(orc, beta):
    """The Gaussian alternative to Eq. Z has the same integral breadth: its
    integral over the support divided by its peak equals that of the Hosemann
    factor over one period (both beta, Eq. breadth); K = exp(-pi t^2/beta^2)/beta
    against the textbook Gaussian integral erf(sqrt(pi) x / beta) beta;
    support min(K_z beta, 1/2)."""
    peak_g = orc.lineshape(2, 0.0, beta)
    peak_h = orc.lineshape(1, 0.0, beta)
    tm = orc.support(2, beta, 3.0)
    assert tm == pytest.approx(min(3.0 * beta, 0.5))
    int_g, _ = si.quad(lambda t: orc.lineshape(2, t, beta), -tm, tm, epsabs=1e-14, epsrel=1e-13, limit=400)
    int_h, _ = si.quad(lambda t: orc.lineshape(1, t, beta), -0.5, 0.5, epsabs=1e-13, epsrel=1e-13, limit=400,
                       points=[0.0])
    assert int_g == pytest.approx(math.erf(math.sqrt(math.pi) * tm / beta), rel=1e-11)
    assert int_g / peak_g == pytest.approx(int_h / peak_h, rel=1e-9 + math.erfc(math.sqrt(math.pi) * tm / beta))
    assert peak_g == pytest.approx(peak_h, rel=1e-13)
    for x in (0.5, 1.0, 2.0):
        assert orc.lineshape(2, x * beta, beta) * beta == pytest.approx(math.exp(-math.pi * x * x), rel=1e-13)


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_lineshape_beta_derivative(orc, kind):
    for beta in (0.05, 0.2, 0.6):
        for t in (0.0, 0.013, 0.07, 0.21, 0.44):
            _, d = orc.lineshape(kind, t, beta, with_derivative=True)
            e = 1e-6 * beta
            fd = (orc.lineshape(kind, t, beta + e) - orc.lineshape(kind, t, beta - e)) / (2 * e)
            assert d == pytest.approx(fd, rel=1e-6, abs=1e-7 * abs(orc.lineshape(kind, 0.0, beta)))


# ------------------------------------------------------------- angular g ---

def test_angular_normalisation_and_fwhm(orc):
    """Sect. Angular peak shapes: g(0) = 1 for all branches; FWHM_G =
    2 sqrt(2 ln 2) sigma ~ 2.3548 sigma, FWHM_L = 2 gamma, ratio ~ 1.177."""
    s = math.radians(3.0)
    assert orc.angular(0.0, s, 0.0) == 1.0
    assert orc.angular(0.0, 0.0, s) == 1.0
    assert orc.angular(0.0, s, 0.5 * s) == pytest.approx(1.0, abs=1e-14)
    import scipy.optimize as so
    hg = so.brentq(lambda d: orc.angular(d, s, 0.0) - 0.5, 0, 5 * s, xtol=1e-15)
    hl = so.brentq(lambda d: orc.angular(d, 0.0, s) - 0.5, 0, 5 * s, xtol=1e-15)
    gold = GOLD
    assert round(2 * hg / s, gold["fwhm_gauss_over_sigma"]["digits"]) == gold["fwhm_gauss_over_sigma"]["value"]
    assert 2 * hl / s == pytest.approx(gold["fwhm_lorentz_over_gamma"]["value"], rel=1e-12)
    ratio = hg / hl
    assert round(ratio, gold["gauss_over_lorentz_fwhm_equal_params"]["digits"]) == \
        gold["gauss_over_lorentz_fwhm_equal_params"]["value"]


@pytest.mark.parametrize("sig_deg,gam_deg", [(3.0, 2.0), (1.0, 4.0), (4.0, 0.3), (0.2, 3.0)])
def test_voigt_against_scipy(orc, sig_deg, gam_deg):
    """The Voigt branch is the normalised convolution (G*L)(d)/(G*L)(0);
    scipy.special.voigt_profile evaluates the same function through the
    Faddeeva function, an independent method."""
    s, g = math.radians(sig_deg), math.radians(gam_deg)
    for d in np.linspace(0.0, 0.5, 23):
        ref = ss.voigt_profile(d, s, g) / ss.voigt_profile(0.0, s, g)
        assert orc.angular(d, s, g) == pytest.approx(ref, rel=2e-12, abs=1e-15)


def test_voigt_limits_and_derivatives(orc):
    """Voigt -> Lorentzian as sigma -> 0 and -> Gaussian as gamma -> 0 (the
    deviation shrinks in proportion to gamma); the sigma/gamma derivatives
    agree with central differences."""
    s = math.radians(2.0)
    for d in (0.0, 0.02, 0.1):
        dev = [orc.angular(d, f * s, s) / orc.angular(d, 0.0, s) - 1.0 for f in (1e-2, 1e-3)]
        assert abs(dev[1]) < 3e-6
        if d > 0:
            assert dev[0] / dev[1] == pytest.approx(100.0, rel=2e-2)  # O(sigma^2) approach
    for d in (s, 2 * s):
        G = orc.angular(d, s, 0.0)
        dev = [orc.angular(d, s, f * s) / G - 1.0 for f in (1e-3, 1e-4, 1e-5)]
        assert dev[0] / dev[1] == pytest.approx(10.0, rel=1e-2)
        assert dev[1] / dev[2] == pytest.approx(10.0, rel=1e-2)
        assert abs(dev[2]) < 3e-5
    for (sg, gm) in ((s, 0.0), (0.0, s), (s, 0.7 * s)):
        for d in (0.0, 0.01, 0.05, 0.12):
            g0, ds, dg = orc.angular(d, sg, gm, with_derivatives=True)
            e = 1e-6
            if sg > 0:
                fd = (orc.angular(d, sg * (1 + e), gm) - orc.angular(d, sg * (1 - e), gm)) / (2 * e * sg)
                assert ds == pytest.approx(fd, rel=1e-5, abs=1e-9)
            if gm > 0:
                fd = (orc.angular(d, sg, gm * (1 + e)) - orc.angular(d, sg, gm * (1 - e))) / (2 * e * gm)
                assert dg == pytest.approx(fd, rel=1e-5, abs=1e-9)


# ---------------------------------------------------------- shell nodes ---

def test_node_weights_solid_angle(orc):
    """Eqs. gnomonic and node_weight with g = 1: sum_k w_k / (sigma_r
    sqrt(2 pi)) is the midpoint rule for the solid angle of the square
    gnomonic patch, 4 asin(T^2 / (1 + T^2)); the error falls as h^2."""
    p = W.small_sinc()
    T = 0.3
    errs = []
    for n in (16, 32, 64):
        d1, d2, w, _, _ = orc.nodes(p, n_nodes=n, T=T, sigma=1e6, gamma=0.0)
        tot = w.sum() / (p.br.sigma_r * math.sqrt(2 * math.pi))
        errs.append(abs(tot - 4 * math.asin(T * T / (1 + T * T))))
        h = 2 * T / n
        assert np.allclose(d1[:, 0], -T + (np.arange(n) + 0.5) * h)
        assert np.allclose(d2[0, :], -T + (np.arange(n) + 0.5) * h)
    assert errs[2] < 1e-4
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.05)


def test_node_weights_gaussian_cap(orc):
    """With a Gaussian shape well inside the patch, the weights integrate g
    over the sphere: 2 pi int_0^{pi/2} exp(-D^2 / 2 s^2) sin D dD."""
    p = W.small_sinc()
    s = math.radians(2.0)
    T = math.tan(12 * s)
    d1, d2, w, _, _ = orc.nodes(p, n_nodes=256, T=T, sigma=s, gamma=0.0)
    tot = w.sum() / (p.br.sigma_r * math.sqrt(2 * math.pi))
    ref, _ = si.quad(lambda D: 2 * math.pi * math.exp(-D * D / (2 * s * s)) * math.sin(D), 0, math.pi / 2,
                     epsabs=1e-15, epsrel=1e-13)
    assert tot == pytest.approx(ref, rel=2e-5)


# ------------------------------------------------------------- geometry ---

def test_pixel_on_ewald_sphere(orc):
    """Eq. laue: every pixel's S satisfies |k_in + S| = 1/lambda; (R, Z) are
    the components of S across and along the fiber axis (tilted or not)."""
    for f in (W.small_sinc, W.small_helix, W.config2, W.small_tilted):
        p = f()
        k_in = np.array(p.geom.beam_axis) / p.geom.wavelength
        n = np.array(p.geom.fiber_axis) / np.linalg.norm(p.geom.fiber_axis)
        for (i, j) in ((0, 0), (p.geom.n_x - 1, 3), (p.geom.n_x // 2, p.geom.n_y // 2), (7, p.geom.n_y - 1)):
            S, R, Z = orc.pixel_S(p, i, j)
            assert np.linalg.norm(k_in + S) == pytest.approx(1.0 / p.geom.wavelength, rel=1e-14)
            assert R == pytest.approx(np.linalg.norm(S - (S @ n) * n), rel=1e-12)
            assert Z == pytest.approx(S @ n, rel=1e-12, abs=1e-16)


def _paper_ewald_solutions(S, n, k_in, lam):
    """Eqs. rodrigues, harmonic and solutions written out from the paper:
    P cos(phi) + Q sin(phi) = R, phi = phi0 +- arccos(R / sqrt(P^2 + Q^2))."""
    A = k_in @ S
    Bq = k_in @ np.cross(n, S)
    Dq = (k_in @ n) * (n @ S)
    Cq = k_in @ k_in + S @ S
    E = ((1.0 / lam) ** 2 - Cq) / 2.0 - Dq
    P, Q, Rr = A - Dq, Bq, E
    ratio = Rr / math.hypot(P, Q)
    if abs(ratio) > 1:
        return []
    phi0 = math.atan2(Q, P)
    out = []
    for sgn in (1, -1):
        phi = phi0 + sgn * math.acos(ratio)
        Sp = S * math.cos(phi) + np.cross(n, S) * math.sin(phi) + n * (n @ S) * (1 - math.cos(phi))
        out.append(Sp)
    return out


@pytest.mark.parametrize("tilt", [0.0, 20.0])
def test_pixel_roundtrip_paper_forward_solver(orc, tilt):
    """Take a pixel's S, rotate it about the fiber axis to a random azimuth,
    and bring it back into the diffraction condition with the paper's closed
    form (Eqs. harmonic, solutions); one of the two solutions must land on
    the same detector pixel (flat detector; fiber axis tilted by `tilt`
    degrees towards the beam)."""
    p = W.tilted(W.small_helix(), tilt) if tilt else W.small_helix()
    n = np.array(p.geom.fiber_axis, dtype=float)
    n /= np.linalg.norm(n)
    b = np.array(p.geom.beam_axis, dtype=float)
    lam = p.geom.wavelength
    u_hat = np.cross(n, b)
    u_hat /= np.linalg.norm(u_hat)
    v_hat = np.cross(b, u_hat)
    rng = np.random.default_rng(11)
    for _ in range(12):
        i, j = int(rng.integers(0, p.geom.n_x)), int(rng.integers(0, p.geom.n_y))
        S, R, Z = orc.pixel_S(p, i, j)
        psi = rng.uniform(0, 2 * math.pi)
        Srot = S * math.cos(psi) + np.cross(n, S) * math.sin(psi) + n * (n @ S) * (1 - math.cos(psi))
        hits = []
        for Sp in _paper_ewald_solutions(Srot, n, b / lam, lam):
            k_out = b / lam + Sp
            t = p.geom.distance / (k_out @ b)
            r = t * k_out
            u, v = r @ u_hat, r @ v_hat
            hits.append((u / p.geom.pixel + p.geom.n_x / 2 - 0.5, v / p.geom.pixel + p.geom.n_y / 2 - 0.5))
        assert any(abs(x - i) < 1e-7 and abs(y - j) < 1e-7 for (x, y) in hits), (i, j, hits)


@pytest.mark.parametrize("delta_L", [1e-5, 1e-2, 1e2])
def test_lorentz_factor(orc, delta_L):
    """Eq. lorentz through the oracle's own composition: for one reflection,
    a pixel's value divided by the reciprocal-space intensity at the pixel's
    query point (oracle.point, which applies no Lorentz factor) is L(R);
    0 < L <= 1, L -> 1 for R << delta_L and L R / delta_L -> 1 for
    R >> delta_L."""
    from dataclasses import replace
    p = W.small_helix()
    p = replace(p, geom=replace(p.geom, delta_L=delta_L))
    hkl_all = orc.reflections(p.cell, p.d_min)
    n = np.array(p.geom.fiber_axis, float) / np.linalg.norm(p.geom.fiber_axis)
    _, As = orc.basis(p.cell)
    As = np.asarray(As)
    pix = orc.all_pixels(p)
    checked = 0
    low = hkl_all[np.argsort(np.linalg.norm(hkl_all @ As, axis=1))][:24]  # the reflections nearest the beam
    for hkl in low:
        one = hkl.reshape(1, 3)
        I, _ = orc.pattern(p, one, np.ones(1), pix)
        hit = np.nonzero(I > 0)[0][:6]
        if len(hit) == 0:
            continue
        D = one[0] @ As
        perp = D - (D @ n) * n
        if np.linalg.norm(perp) < 1e-12:
            continue  # meridional reflection: e_R is the frame's e1, covered elsewhere
        eR = perp / np.linalg.norm(perp)
        for q in hit:
            _, R, Z = orc.pixel_S(p, int(pix[q, 0]), int(pix[q, 1]))
            Ip = orc.point(p, one, np.ones(1), (Z * n + R * eR).reshape(1, 3))[0]
            L = I[q] / Ip
            assert L == pytest.approx(delta_L / (R + delta_L), rel=1e-10)
            assert 0.0 < L <= 1.0
            if R < 1e-3 * delta_L:
                assert L > 0.999
            if R > 1e3 * delta_L:
                assert L * R / delta_L == pytest.approx(1.0, rel=2e-3)
            checked += 1
    assert checked >= 20
