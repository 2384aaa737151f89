"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle on the
same seeded inputs.  Gates (per result): max |dI| <= 1e-5 max I_oracle and
||dI||_2 <= 1e-6 ||I_oracle||_2 for the pattern; the in-support term count of
every pixel lies between the oracle's counts with the support shrunk and
grown by 1e-6 (the decision is taken in FP32 on the GPU and in FP64 by the
oracle, so only terms within rounding of the support edge may differ)."""
import math
from dataclasses import replace

import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W
from _common import L2_REL, MAX_REL, SF_TOL, amp_scale as _amp_scale, api_precision, oracle_hkl, parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2608_23245_b300 import _build, fdx
    _build.build()
    return fdx


SMALL = [W.small_sinc, W.small_helix, W.small_lorentz, W.small_triclinic, W.small_gauss, W.small_tilted]


def _sync():
    import torch
    torch.cuda.synchronize()


def test_reflections_device_buffer(gpu, orc):
    import ctypes as C
    import torch
    for make in (W.config0, W.config1, W.small_triclinic):
        p = make()
        ref = orc.reflections(p.cell, p.d_min)
        buf = torch.zeros((len(ref), 3), dtype=torch.int32, device="cuda")
        n = C.c_int32(0)
        cell = gpu.make_cell(p.cell)
        rc = gpu.lib().fdx_reflections(C.byref(cell), p.d_min, p.d_max, len(ref), C.c_void_p(buf.data_ptr()),
                                       C.byref(n))
        assert rc == 0 and n.value == len(ref)
        assert np.array_equal(buf.cpu().numpy(), ref)


@pytest.mark.parametrize("make", SMALL + [W.config0, W.config1])
def test_structure_factors(gpu, orc, make):
    """Eq. structure_factor: |F_gpu - F_oracle| <= 2e-6 sqrt(sum_j amp_j^2)
    per reflection, and M = |F|^2 P DW within the same relative budget."""
    p = api_precision(make())
    sim = gpu.Simulation(p)
    F, M = sim.structure_factors()
    _sync()
    F = F.cpu().numpy().astype(np.float64)
    Fg = F[:, 0] + 1j * F[:, 1]
    hkl = oracle_hkl(orc, p, sim.hkl_host)
    Fo = orc.structure_factors(p.cell, p.atoms, hkl)
    Mo = orc.intensities_M(p, hkl, Fo)
    scale = _amp_scale(p, hkl)
    err = np.abs(Fg - Fo) / scale
    assert err.max() <= SF_TOL, err.max()
    Mg = M.cpu().numpy().astype(np.float64)
    _, P, DW = orc.refl_scalars(p, hkl)
    merr = np.abs(Mg - Mo) / ((2 * np.abs(Fo) + scale) * scale * P * DW)
    assert merr.max() <= 4e-6, merr.max()


def test_structure_factors_large_subset(gpu, orc):
    """The 20,000-atom cell on a seeded 3,000-reflection subset of d >= 1.5 A."""
    import torch
    p = api_precision(W.config2())
    hkl_all = gpu.fdx_reflections(p.cell, p.d_min)
    rng = np.random.default_rng(2608)
    hkl = hkl_all[np.sort(rng.choice(len(hkl_all), 3000, replace=False))]
    atoms = gpu.DeviceAtoms(p.atoms)
    F, _ = gpu.fdx_structure_factors(p.cell, atoms, torch.as_tensor(hkl, device="cuda"), p.br)
    _sync()
    Fg = F.cpu().numpy().astype(np.float64)
    Fg = Fg[:, 0] + 1j * Fg[:, 1]
    Fo = orc.structure_factors(p.cell, p.atoms, hkl)
    err = np.abs(Fg - Fo) / _amp_scale(p, hkl)
    assert err.max() <= SF_TOL, err.max()


def _many_elements(p, n_elem=48, seed=4811):
    """p's atoms re-typed over n_elem element types (more than one pass of the
    form-factor table), a few types left without atoms, occupancies in
    {0, 0.5, 1}: every element run of the sorted atom list has a ragged tail."""
    rng = np.random.default_rng(seed)
    a = p.atoms
    n = a.n
    used = np.setdiff1d(np.arange(n_elem), [3, 17, 41, 47])
    elem = rng.choice(used, size=n).astype(np.uint8)
    ff = np.concatenate([rng.uniform(0.5, 3.0, (n_elem, 4)), rng.uniform(0.5, 40.0, (n_elem, 4)),
                         rng.uniform(0.0, 1.0, (n_elem, 1))], axis=1)
    occ = rng.choice([0.0, 0.5, 1.0], size=n, p=[0.1, 0.2, 0.7])
    return api_precision(replace(p, atoms=replace(a, elem=elem, ff=ff, occ=occ)))


@pytest.mark.parametrize("make", [W.small_helix, W.config1])
def test_structure_factors_many_elements(gpu, orc, make):
    """48 element types (two passes of the form-factor table), unused types
    and partial occupancies, against the oracle with the same tolerance."""
    import torch
    p = _many_elements(make())
    hkl = gpu.fdx_reflections(p.cell, p.d_min)
    atoms = gpu.DeviceAtoms(p.atoms)
    F, _ = gpu.fdx_structure_factors(p.cell, atoms, torch.as_tensor(hkl, device="cuda"), p.br)
    _sync()
    Fg = F.cpu().numpy().astype(np.float64)
    Fg = Fg[:, 0] + 1j * Fg[:, 1]
    Fo = orc.structure_factors(p.cell, p.atoms, hkl)
    err = np.abs(Fg - Fo) / _amp_scale(p, hkl)
    assert err.max() <= SF_TOL, err.max()


def test_structure_factors_bad_element_is_nan(gpu):
    """An element index >= n_elem poisons every F with NaN (documented)."""
    import torch
    p = api_precision(W.small_helix())
    elem = p.atoms.elem.copy()
    elem[37] = p.atoms.ff.shape[0]
    p = replace(p, atoms=replace(p.atoms, elem=elem))
    hkl = gpu.fdx_reflections(p.cell, p.d_min)
    F, _ = gpu.fdx_structure_factors(p.cell, gpu.DeviceAtoms(p.atoms), torch.as_tensor(hkl, device="cuda"), p.br)
    _sync()
    assert torch.isnan(F).all()


def test_structure_factors_edge_cases(gpu, orc):
    """One atom (F = occ f(s) exp(-B s^2/4), the closed form of Eq.
    structure_factor for a single atom at the origin), zero occupancy (F = 0),
    an empty reflection list (no work, no error), and 1,025 atoms (a ragged
    second chunk of the element sort)."""
    import torch
    p = api_precision(W.small_helix())
    hkl = gpu.fdx_reflections(p.cell, p.d_min)
    hk = torch.as_tensor(hkl, device="cuda")
    a = p.atoms
    one = replace(a, frac=np.zeros((1, 3)), B=np.array([12.0]), occ=np.array([0.75]), elem=np.array([2], np.uint8))
    one = api_precision(replace(p, atoms=one)).atoms
    F, _ = gpu.fdx_structure_factors(p.cell, gpu.DeviceAtoms(one), hk, p.br)
    _sync()
    _, As = orc.basis(p.cell)
    s2 = np.sum((hkl.astype(np.float64) @ np.asarray(As).reshape(3, 3)) ** 2, axis=1)
    ff = one.ff[2]
    f = ff[8] + np.sum(ff[None, 0:4] * np.exp(-ff[None, 4:8] * s2[:, None] / 4), axis=1)
    ref = one.occ[0] * f * np.exp(-one.B[0] * s2 / 4)
    Fg = F.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(Fg[:, 0] - ref)) <= 2e-6 * np.max(ref) and np.max(np.abs(Fg[:, 1])) <= 2e-6 * np.max(ref)
    zero = replace(a, occ=np.zeros(a.n))
    F0, _ = gpu.fdx_structure_factors(p.cell, gpu.DeviceAtoms(zero), hk, p.br)
    _sync()
    assert torch.all(F0 == 0)
    Fe, Me = gpu.fdx_structure_factors(p.cell, gpu.DeviceAtoms(a), hk[:0], p.br)
    _sync()
    assert Fe.numel() == 0 and Me.numel() == 0
    rng = np.random.default_rng(1025)
    big = api_precision(replace(p, atoms=replace(a, frac=rng.uniform(0, 1, (1025, 3)), B=rng.uniform(10, 30, 1025),
                                                 occ=np.ones(1025), elem=rng.integers(0, 4, 1025).astype(np.uint8))))
    Fb, _ = gpu.fdx_structure_factors(p.cell, gpu.DeviceAtoms(big.atoms), hk, p.br)
    _sync()
    Fb = Fb.cpu().numpy().astype(np.float64)
    Fo = orc.structure_factors(p.cell, big.atoms, hkl)
    err = np.abs(Fb[:, 0] + 1j * Fb[:, 1] - Fo) / _amp_scale(big, hkl)
    assert err.max() <= SF_TOL, err.max()


def _gpu_pattern(gpu, p, hkl, M):
    import torch
    hk = torch.as_tensor(np.ascontiguousarray(hkl, np.int32), device="cuda").reshape(-1, 3)
    Mt = torch.as_tensor(np.ascontiguousarray(M, np.float32), device="cuda")
    prob = gpu.make_problem(p.cell, p.br, p.geom, hk, Mt)
    img = torch.empty((p.geom.n_y, p.geom.n_x), dtype=torch.float32, device="cuda")
    gpu.fdx_pattern([prob], [img])
    cnt = torch.empty((p.geom.n_y, p.geom.n_x), dtype=torch.int32, device="cuda")
    gpu.fdx_pattern_evals(prob, cnt)
    _sync()
    return img.cpu().numpy(), cnt.cpu().numpy()


@pytest.mark.parametrize("make", SMALL + [W.config0])
def test_pattern_full_image(gpu, orc, make):
    """Whole detector, intensities M from the oracle (rounded to float32 as
    the C-ABI takes them): isolates the pattern kernel."""
    p = api_precision(make())
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl).astype(np.float32)
    I, E = orc.pattern(p, hkl, M.astype(np.float64))
    img, cnt = _gpu_pattern(gpu, p, hkl, M)
    mr, l2 = parity(img.reshape(-1), I)
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)
    c = cnt.reshape(-1)
    assert np.all(c >= E[:, 1]) and np.all(c <= E[:, 2]), (int(np.sum(c < E[:, 1])), int(np.sum(c > E[:, 2])))


@pytest.mark.parametrize("make", [W.small_helix, W.small_triclinic, W.config0])
def test_end_to_end(gpu, orc, make):
    """Structure factors and pattern on the GPU against the oracle's
    structure factors and pattern."""
    p = api_precision(make())
    sim = gpu.Simulation(p)
    img = sim.forward()
    _sync()
    img = img.cpu().numpy()
    hkl = oracle_hkl(orc, p, sim.hkl_host)
    Mo = orc.intensities_M(p, hkl)
    I, _ = orc.pattern(p, hkl, Mo)
    mr, l2 = parity(img.reshape(-1), I)
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)


def test_helix_full_size_sampled(gpu, orc):
    """The 2,000-atom helix at full size (1024^2 detector, 64^2 nodes), in the
    launch configuration the benchmark times, on 96 seeded pixels: 48 drawn
    over the whole detector and 48 from its central quarter."""
    p = api_precision(W.config1())
    sim = gpu.Simulation(p)
    img = sim.forward()
    cnt = sim.evals()
    _sync()
    img, cnt = img.cpu().numpy(), cnt.cpu().numpy()
    rng = np.random.default_rng(26082)
    n = p.geom.n_x
    ii = np.concatenate([rng.integers(0, n, 48), rng.integers(n // 4, 3 * n // 4, 48)])
    jj = np.concatenate([rng.integers(0, n, 48), rng.integers(n // 4, 3 * n // 4, 48)])
    pix = np.stack([ii, jj], axis=1).astype(np.int32)
    hkl = oracle_hkl(orc, p, sim.hkl_host)
    Mo = orc.intensities_M(p, hkl)
    I, E = orc.pattern(p, hkl, Mo, pix)
    got = img[jj, ii]
    mr, l2 = parity(got, I)
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)
    c = cnt[jj, ii]
    assert np.all(c >= E[:, 1]) and np.all(c <= E[:, 2])


@pytest.mark.parametrize("g", [0.01, 0.04])
def test_large_cell_sampled(gpu, orc, g):
    """The 50x50x70 A cell, 20,000 atoms, 128^2 nodes, 2048^2 detector: 8
    seeded pixels in the |S| band [0.30, 0.31] 1/A; intensities of the
    reflections that can reach the band come from the oracle (others 0)."""
    p = api_precision(W.config2(g))
    hkl = orc.reflections(p.cell, p.d_min)
    _, As = orc.basis(p.cell)
    r0 = np.linalg.norm(hkl @ As, axis=1)
    near = np.abs(r0 - 0.305) < 0.03
    M = np.zeros(len(hkl), np.float32)
    M[near] = orc.intensities_M(p, hkl[near]).astype(np.float32)
    rng = np.random.default_rng(int(g * 1000) + 7)
    pix = []
    while len(pix) < 8:
        i, j = (int(x) for x in rng.integers(0, p.geom.n_x, 2))
        _, R, Z = orc.pixel_S(p, i, j)
        if 0.30 <= math.hypot(R, Z) <= 0.31:
            pix.append((i, j))
    pix = np.array(pix, np.int32)
    I, E = orc.pattern(p, hkl, M.astype(np.float64), pix)
    img, cnt = _gpu_pattern(gpu, p, hkl, M)
    got = img[pix[:, 1], pix[:, 0]]
    mr, l2 = parity(got, I)
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)
    c = cnt[pix[:, 1], pix[:, 0]]
    assert np.all(c >= E[:, 1]) and np.all(c <= E[:, 2])


def test_edge_cases(gpu, orc):
    """Empty reflection list, 1x1 and ragged detectors, a meridional-only
    list (e_R = e1 branch) and reflections smaller than their support box."""
    p = api_precision(W.small_triclinic())
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl).astype(np.float32)
    img, cnt = _gpu_pattern(gpu, p, hkl[:0], M[:0])
    assert np.all(img == 0) and np.all(cnt == 0)
    for nx, ny in ((1, 1), (17, 9), (33, 5)):
        q = replace(p, geom=replace(p.geom, n_x=nx, n_y=ny, pixel=p.geom.pixel * 64 / nx))
        I, _ = orc.pattern(q, hkl, M.astype(np.float64))
        img, _ = _gpu_pattern(gpu, q, hkl, M)
        mr, l2 = parity(img.reshape(-1), I)
        assert mr <= MAX_REL and l2 <= L2_REL, (nx, ny, mr, l2)
    mer = hkl[(hkl[:, 0] == 0) & (hkl[:, 1] == 0)]
    Mm = orc.intensities_M(p, mer).astype(np.float32)
    I, _ = orc.pattern(p, mer, Mm.astype(np.float64))
    img, _ = _gpu_pattern(gpu, p, mer, Mm)
    assert I.max() > 0
    mr, l2 = parity(img.reshape(-1), I)
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)
    # a coarse cell whose lowest orders lie inside their own support box
    q = replace(p, br=replace(p.br, L=(15.0, 15.0, 15.0)), d_min=6.0)
    h2 = orc.reflections(q.cell, q.d_min)
    M2 = orc.intensities_M(q, h2).astype(np.float32)
    I, E = orc.pattern(q, h2, M2.astype(np.float64))
    img, cnt = _gpu_pattern(gpu, q, h2, M2)
    mr, l2 = parity(img.reshape(-1), I)
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)


def test_deterministic(gpu):
    """No atomics: two runs give bitwise identical images and F."""
    import torch
    p = api_precision(W.small_helix())
    sim = gpu.Simulation(p)
    a = sim.forward().clone()
    F1 = sim.F.clone()
    b = sim.forward().clone()
    _sync()
    assert torch.equal(a, b)
    assert torch.equal(F1, sim.F)


def test_mirror_symmetry_gpu(gpu):
    """Meridian and equator mirror symmetry of the GPU image (to rounding)."""
    p = api_precision(W.small_lorentz())
    sim = gpu.Simulation(p)
    img = sim.forward()
    _sync()
    img = img.cpu().numpy().astype(np.float64)
    s = img.max()
    assert np.max(np.abs(img - img[:, ::-1])) <= 2e-6 * s
    assert np.max(np.abs(img - img[::-1, :])) <= 2e-6 * s


def test_status_after_work(gpu):
    """fdx_status on the stream of a finished forward pass: success, code 0."""
    p = api_precision(W.small_helix())
    sim = gpu.Simulation(p)
    sim.forward()
    assert gpu.fdx_status() == 0


@pytest.mark.parametrize("n_nodes", [1, 2, 7, 33, 130, 257, 512])
def test_node_grid_sizes(gpu, orc, n_nodes):
    """Node grids from one node to 512 per axis (ragged culling blocks,
    bounding boxes clipped by the grid's edge, many flushes of the staging
    buffers) on a small ragged detector: whole-image parity and the in-support
    count bracket."""
    p = api_precision(W.small_helix())
    p = replace(p, br=replace(p.br, n_nodes=n_nodes), geom=replace(p.geom, n_x=17, n_y=13))
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl).astype(np.float32)
    I, E = orc.pattern(p, hkl, M.astype(np.float64))
    img, cnt = _gpu_pattern(gpu, p, hkl, M)
    assert I.max() > 0
    mr, l2 = parity(img.reshape(-1), I)
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)
    c = cnt.reshape(-1)
    assert np.all(c >= E[:, 1]) and np.all(c <= E[:, 2])


def test_pattern_several_models_one_call(gpu, orc):
    """fdx_pattern over three different problems in one call (one workspace
    of the largest model's size, reused in stream order) gives each model's
    single-call image bit for bit."""
    import torch
    probs, imgs, refs, keep = [], [], [], []
    for make in (W.small_helix, W.small_triclinic, W.small_sinc):
        p = api_precision(make())
        hkl = orc.reflections(p.cell, p.d_min)
        M = orc.intensities_M(p, hkl).astype(np.float32)
        refs.append(_gpu_pattern(gpu, p, hkl, M)[0])
        hk = torch.as_tensor(np.ascontiguousarray(hkl, np.int32), device="cuda").reshape(-1, 3)
        Mt = torch.as_tensor(M, device="cuda")
        keep += [hk, Mt]
        probs.append(gpu.make_problem(p.cell, p.br, p.geom, hk, Mt))
        imgs.append(torch.full((p.geom.n_y, p.geom.n_x), float("nan"), dtype=torch.float32, device="cuda"))
    gpu.fdx_pattern(probs, imgs)
    _sync()
    for img, ref in zip(imgs, refs):
        assert np.array_equal(img.cpu().numpy(), ref)
