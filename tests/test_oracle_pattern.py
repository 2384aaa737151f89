"""Pins for the oracle's pattern and adjoint (Eqs. shell_conv, gnomonic,
node_weight, direct_sum, lorentz), against invariants, limits, an
independent quadrature of the shell convolution, and finite differences."""
import math
from dataclasses import replace

import numpy as np
import pytest
import scipy.integrate as si

from paper_2608_23245_b300 import workloads as W


def _frame(As, hkl, n, b):
    """Reflection frame of reading R9 and the query-point direction of R12."""
    D = np.asarray(hkl, float) @ As
    r0 = np.linalg.norm(D)
    Sh = D / r0
    e1 = np.cross(n, Sh)
    if np.linalg.norm(e1) < 1e-12:
        e1 = np.cross(b, Sh)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(Sh, e1)
    ZD = D @ n
    perp = D - ZD * n
    eR = perp / np.linalg.norm(perp) if np.linalg.norm(perp) > 1e-12 * r0 else e1
    return D, r0, Sh, e1, e2, eR


def _single(p, hkl, r):
    M = np.zeros(len(hkl))
    M[r] = 1.0
    return M


@pytest.mark.parametrize("make", [W.small_sinc, W.small_triclinic, W.small_gauss])
def test_cull_is_exact(orc, make):
    """Skipping reflections with | |p| - r0 | > rho_B changes nothing."""
    p = make()
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl)
    pix = orc.all_pixels(p)[::7]
    I1, E1 = orc.pattern(p, hkl, M, pix, cull=True)
    I0, E0 = orc.pattern(p, hkl, M, pix, cull=False)
    assert np.array_equal(I1, I0)
    assert np.array_equal(E1, E0)


@pytest.mark.parametrize("make", [W.small_sinc, W.small_lorentz, W.small_triclinic, W.small_gauss])
def test_mirror_symmetry(orc, make):
    """Fiber symmetry: a pixel and its mirror about the meridian (u -> -u)
    have the same (R, Z), hence the same value; with Friedel-symmetric
    intensities the equator (v -> -v) is a mirror too (inversion S -> -S)."""
    p = make()
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl)
    I, E = orc.pattern(p, hkl, M)
    nx, ny = p.geom.n_x, p.geom.n_y
    img = I.reshape(ny, nx)
    scale = img.max()
    assert scale > 0
    assert np.max(np.abs(img - img[:, ::-1])) <= 1e-12 * scale
    assert np.max(np.abs(img - img[::-1, :])) <= 1e-12 * scale
    cnt = E[:, 0].reshape(ny, nx)
    assert np.array_equal(cnt, cnt[:, ::-1])


def test_mirror_symmetry_tilted(orc):
    """With the fiber axis tilted towards the beam the setup is still mirror
    symmetric about the plane of beam and fiber axis (u -> -u), but not about
    the equator."""
    p = W.small_tilted()
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl)
    I, E = orc.pattern(p, hkl, M)
    img = I.reshape(p.geom.n_y, p.geom.n_x)
    scale = img.max()
    assert scale > 0
    assert np.max(np.abs(img - img[:, ::-1])) <= 1e-12 * scale
    assert np.max(np.abs(img - img[::-1, :])) > 1e-3 * scale


def test_delta_limit(orc):
    """As the orientation spread and patch shrink to a point (sigma -> 0,
    T = tan 3 sigma), the pixel value tends to
    L(R) M r0^2 (sum_k w_k) prod_i K_i(a_i . (p - D)).  Checked for a general
    and a meridional reflection."""
    p = W.small_triclinic()
    sig = 1e-5
    p = replace(p, br=replace(p.br, sigma=sig, gamma=0.0, T=math.tan(3 * sig), n_nodes=6))
    hkl = orc.reflections(p.cell, p.d_min)
    A, As = orc.basis(p.cell)
    beta, _, _ = orc.refl_scalars(p, hkl)
    n = np.array(p.geom.fiber_axis, float)
    b = np.array(p.geom.beam_axis, float)
    _, _, w, _, _ = orc.nodes(p)
    pix = orc.all_pixels(p)
    checked = 0
    for target in ((1, 1, 1), (0, 0, 2)):
        r = int(np.where((hkl == np.array(target)).all(axis=1))[0][0])
        I, _ = orc.pattern(p, hkl, _single(p, hkl, r), pix)
        D, r0, Sh, e1, e2, eR = _frame(As, hkl[r], n, b)
        for q in np.argsort(I)[::-1][:40]:
            S, R, Z = orc.pixel_S(p, *pix[q])
            pq = Z * n + R * eR
            t = A @ (pq - D)
            tm = [orc.support(p.br.lineshape, beta[r, i], p.br.K_z) for i in range(3)]
            if any(abs(t[i]) > tm[i] - 1e-3 for i in range(3)):
                continue
            K = np.prod([orc.lineshape(p.br.lineshape, t[i], beta[r, i]) for i in range(3)])
            L = p.geom.delta_L / (R + p.geom.delta_L)
            ref = L * r0 * r0 * w.sum() * K
            assert I[q] == pytest.approx(ref, rel=1e-6)
            checked += 1
    assert checked >= 20


def test_shell_integral_independent_quadrature(orc):
    """Eq. shell_conv reduced to the surface integral (Sect. Numerical
    evaluation): sigma_r sqrt(2 pi) r0^2 \\int g(Delta) prod K dOmega.  The
    oracle's gnomonic midpoint sum (Eqs. gnomonic, node_weight) must converge
    as h^2 to the same integral computed here in spherical coordinates about
    the query direction with adaptive quadrature."""
    p = W.small_sinc()
    p = replace(p, br=replace(p.br, L=(60.0, 60.0, 90.0)))
    hkl = orc.reflections(p.cell, p.d_min)
    A, As = orc.basis(p.cell)
    beta, _, _ = orc.refl_scalars(p, hkl)
    n = np.array(p.geom.fiber_axis, float)
    b = np.array(p.geom.beam_axis, float)
    r = int(np.where((hkl == np.array([1, 0, 1])).all(axis=1))[0][0])
    M = _single(p, hkl, r)
    pix_all = orc.all_pixels(p)
    I0, _ = orc.pattern(p, hkl, M, pix_all)
    assert I0.max() > 0
    q = int(np.argmax(I0))
    pix = pix_all[q:q + 1]
    vals = []
    for nn in (128, 256, 512):
        I, _ = orc.pattern(p, hkl, M, pix, n_nodes=nn)
        vals.append(I[0])
    ratio = (vals[1] - vals[0]) / (vals[2] - vals[1])
    richardson = vals[2] + (vals[2] - vals[1]) / 3.0

    D, r0, Sh, e1, e2, eR = _frame(As, hkl[r], n, b)
    S, R, Z = orc.pixel_S(p, *pix[0])
    pq = Z * n + R * eR
    ph = pq / np.linalg.norm(pq)
    f1 = np.cross(ph, e1)
    f1 /= np.linalg.norm(f1)
    f2 = np.cross(ph, f1)
    tm = np.array([orc.support(0, beta[r, i], p.br.K_z) for i in range(3)])
    rhoB = max(np.linalg.norm(tm[0] * As[0] + sb * tm[1] * As[1] + sc * tm[2] * As[2])
               for sb in (1, -1) for sc in (1, -1))
    alpha = math.asin(min(1.0, 1.05 * (rhoB + abs(np.linalg.norm(pq) - r0)) / r0))
    sig = p.br.sigma

    def integrand(th, ps):
        nh = math.cos(th) * ph + math.sin(th) * (math.cos(ps) * f1 + math.sin(ps) * f2)
        c = nh @ Sh
        d1, d2 = (nh @ e1) / c, (nh @ e2) / c
        if abs(d1) > p.br.T or abs(d2) > p.br.T:
            return 0.0
        t = A @ (pq - r0 * nh)
        if np.any(np.abs(t) > tm):
            return 0.0
        K = 1.0
        for i in range(3):
            K *= orc.lineshape(0, t[i], beta[r, i])
        Delta = math.acos(min(1.0, c))
        return math.exp(-Delta * Delta / (2 * sig * sig)) * K * math.sin(th)

    val, err = si.dblquad(integrand, 0.0, 2 * math.pi, 0.0, alpha, epsabs=0, epsrel=1e-9)
    Lf = p.geom.delta_L / (R + p.geom.delta_L)
    ref = Lf * r0 * r0 * p.br.sigma_r * math.sqrt(2 * math.pi) * val
    assert ratio == pytest.approx(4.0, rel=0.1)
    assert richardson == pytest.approx(ref, rel=2e-6)
    assert vals[2] == pytest.approx(ref, rel=2e-3)


def _tiny_problem():
    p = W.small_triclinic()
    br = replace(p.br, n_nodes=10)
    geom = replace(p.geom, n_x=30, n_y=22, pixel=1.2)
    atoms = W.Atoms(frac=p.atoms.frac[:12].copy(), B=p.atoms.B[:12].copy(), occ=p.atoms.occ[:12].copy(),
                    elem=p.atoms.elem[:12].copy(), ff=8000.0 * p.atoms.ff)
    return replace(p, br=br, geom=geom, atoms=atoms, d_min=4.0)


def _loss(orc, p, hkl, It):
    M = orc.intensities_M(p, hkl)
    I, _ = orc.pattern(p, hkl, M)
    return orc.loss_and_grad(I, It)[0]


@pytest.mark.parametrize("lineshape", [W.LINESHAPE_HOSEMANN, W.LINESHAPE_SINC, W.LINESHAPE_GAUSS])
def test_adjoint_against_central_differences(orc, lineshape):
    """The oracle's analytic adjoint (pattern -> M, beta, weights -> atoms,
    sizes, g, sigma, gamma) against FP64 central differences of its own
    forward loss L = sum w (I - I_t)^2, w = 1/(I_t + 1), for each lineshape
    (Eq. Z; Eq. I_shape with N = 1/beta, whose support edge K_z/N moves with
    beta but where K and dK/dt vanish; the Gaussian of equal breadth)."""
    p = _tiny_problem()
    if lineshape != W.LINESHAPE_HOSEMANN:
        p = replace(p, br=replace(p.br, lineshape=lineshape))
    hkl = orc.reflections(p.cell, p.d_min)
    rng = np.random.default_rng(1)
    tgt = replace(p, atoms=replace(p.atoms, frac=p.atoms.frac + rng.uniform(-0.01, 0.01, p.atoms.frac.shape)),
                  br=replace(p.br, sigma=p.br.sigma * 1.1, g=tuple(1.2 * x for x in p.br.g)))
    Mt = orc.intensities_M(tgt, hkl)
    It, _ = orc.pattern(tgt, hkl, Mt)
    assert It.max() > 0.5  # form factors scaled so that w = 1/(I_t + 1) varies
    p = replace(p, atoms=p.atoms)
    loss, grads, I = orc.full_gradient(p, hkl, It)

    def fd(setter, x0, h):
        lp = _loss(orc, setter(x0 + h), hkl, It)
        lm = _loss(orc, setter(x0 - h), hkl, It)
        return (lp - lm) / (2 * h)

    checks = []
    for j in (0, 5):
        for c in range(3):
            def set_frac(v, j=j, c=c):
                f = p.atoms.frac.copy()
                f[j, c] = v
                return replace(p, atoms=replace(p.atoms, frac=f))
            checks.append((grads["frac"][j, c], fd(set_frac, p.atoms.frac[j, c], 1e-6)))
        def set_B(v, j=j):
            B = p.atoms.B.copy()
            B[j] = v
            return replace(p, atoms=replace(p.atoms, B=B))
        checks.append((grads["B"][j], fd(set_B, p.atoms.B[j], 1e-4)))
    for i in range(3):
        def set_L(v, i=i):
            L = list(p.br.L)
            L[i] = v
            return replace(p, br=replace(p.br, L=tuple(L)))
        checks.append((grads["L"][i], fd(set_L, p.br.L[i], 1e-5 * p.br.L[i])))
        def set_g(v, i=i):
            g = list(p.br.g)
            g[i] = v
            return replace(p, br=replace(p.br, g=tuple(g)))
        checks.append((grads["g"][i], fd(set_g, p.br.g[i], 1e-6)))
    checks.append((grads["sigma"], fd(lambda v: replace(p, br=replace(p.br, sigma=v)), p.br.sigma, 1e-7)))
    checks.append((grads["gamma"], fd(lambda v: replace(p, br=replace(p.br, gamma=v)), p.br.gamma, 1e-7)))
    scale = max(abs(a) for a, _ in checks)
    for a, f in checks:
        assert a == pytest.approx(f, rel=1e-6, abs=1e-9 * scale)


def test_edge_term_magnitude_marks_exactly_the_ambiguous_pixels(orc):
    """The oracle's edge-term magnitude A (terms whose inclusion flips between
    the support shrunk and grown by eta) is zero exactly where the strict and
    loose counts agree, positive where they differ, and grows with eta (a
    wider band holds at least the same terms); I and E are unchanged by asking
    for it."""
    p = W.small_helix()
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl)
    I0, E0 = orc.pattern(p, hkl, M)
    for eta in (1e-3, 1e-2):
        I, E, A = orc.pattern(p, hkl, M, eta=eta, with_ambiguous=True)
        assert np.array_equal(I, I0) and np.array_equal(E[:, 0], E0[:, 0])
        amb = E[:, 2] > E[:, 1]
        assert amb.any() and np.all(A >= 0)
        assert np.all((A > 0) == amb)
    _, _, A1 = orc.pattern(p, hkl, M, eta=1e-3, with_ambiguous=True)
    _, _, A2 = orc.pattern(p, hkl, M, eta=1e-2, with_ambiguous=True)
    assert np.all(A2 >= A1) and A2.sum() > A1.sum()
