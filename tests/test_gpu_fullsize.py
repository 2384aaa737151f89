"""Parity at the workloads' full sizes, in the launch configurations the
benchmark times.

- Large forward (20,000 atoms, 217,252 reflections, 128^2 nodes, 2048^2
  detector; g = 1 % and 4 %): the GPU's structure factors and pattern, end to
  end, against the FP64 oracle's at 1,024 seeded pixels over the whole
  detector plus the full meridian column and equator row.  The oracle values
  come from tests/golden/make_config2_samples.py (oracle only), stored with a
  fingerprint of the inputs.  Where a pixel has terms within rounding of the
  lineshape support's edge (FP32 here, FP64 in the oracle) it has two correct
  values; those pixels are bounded by the magnitude of their edge terms.
- Batched refinement: eight real models of the 256-model recipe (the one with
  the most atoms, the one with the largest detector, six seeded others),
  through fdx_batch_refine with a 256-pixel mask, against the oracle's forward
  at those pixels and the oracle's full adjoint of the masked loss.

Gates as elsewhere: max |dI| <= 1e-5 max I, ||dI||_2 <= 1e-6 ||I||_2, counts
within the oracle's strict/loose bracket, gradients within 1e-4."""
import os
import sys

import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W
from _common import L2_REL, MAX_REL, api_precision, oracle_hkl, parity

pytestmark = pytest.mark.gpu

ADJ_TOL = 1e-4
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2608_23245_b300 import _build, fdx
    _build.build()
    return fdx


def _samples():
    sys.path.insert(0, GOLDEN)
    import make_config2_samples as mk
    return mk, np.load(os.path.join(GOLDEN, "config2_oracle_samples.npz"))


@pytest.mark.parametrize("g", [0.01, 0.04])
def test_large_forward_full_size(gpu, g):
    import torch
    mk, data = _samples()
    key = "g%d" % round(1000 * g)
    p = mk.problem(g)
    sim = gpu.Simulation(p)
    pix = data["pix"]
    assert str(data[key + "_fp"]) == mk.fingerprint(p, sim.hkl_host, pix), "stale oracle samples: regenerate them"
    img = sim.forward()
    cnt = sim.evals()
    torch.cuda.synchronize()
    img, cnt = img.cpu().numpy(), cnt.cpu().numpy()
    I, E, A = data[key + "_I"], data[key + "_E"], data[key + "_A"]
    ii, jj = pix[:, 0], pix[:, 1]
    got = img[jj, ii].astype(np.float64)
    # A pixel with terms within rounding of the support's edge (the Hosemann
    # factor is beta, not zero, at |t| = 1/2, so each such term is a jump) has
    # two correct values, the kernel deciding in FP32 and the oracle in FP64;
    # every other pixel has one.  Unambiguous pixels: the gates (max per line
    # of pixels, L2 over the whole sample).  Ambiguous ones: off by at most the
    # magnitude of their edge terms.
    one = A == 0.0
    err = np.abs(got - I)
    n_rand = len(pix) - p.geom.n_x - p.geom.n_y
    for name, sl in (("random", slice(0, n_rand)), ("meridian", slice(n_rand, n_rand + p.geom.n_y)),
                     ("equator", slice(n_rand + p.geom.n_y, len(pix)))):
        mx = np.abs(I[sl]).max()
        assert mx > 0 and one[sl].mean() > 0.5, (name, one[sl].mean())
        assert err[sl][one[sl]].max() <= MAX_REL * mx, (name, err[sl][one[sl]].max() / mx)
        assert np.all(err[sl] <= A[sl] + MAX_REL * mx), (name, np.max(err[sl] - A[sl]) / mx)
    l2 = np.linalg.norm(err[one]) / np.linalg.norm(I[one])
    assert l2 <= L2_REL, l2
    c = cnt[jj, ii]
    assert np.all(c >= E[:, 1]) and np.all(c <= E[:, 2]), (int(np.sum(c < E[:, 1])), int(np.sum(c > E[:, 2])))
    assert int(E[:, 0].sum()) > 10 ** 8


def _chosen_models():
    sizes = []
    for m in range(256):
        q = W.config4_model(m)
        sizes.append((q.atoms.n, q.geom.n_x))
    sizes = np.array(sizes)
    first = [int(np.argmax(sizes[:, 0])), int(np.argmax(sizes[:, 1]))]
    rng = np.random.default_rng(4096)
    rest = [int(m) for m in rng.permutation(256) if m not in first][:6]
    return first + rest


def test_batched_real_models(gpu, orc):
    import torch
    chosen = _chosen_models()
    models = [api_precision(W.config4_model(m)) for m in chosen]
    sims = [gpu.Simulation(p) for p in models]
    rng = np.random.default_rng(4097)
    pixes, Io, Eo, Its, targets, masks = [], [], [], [], [], []
    for p, s in zip(models, sims):
        n = p.geom.n_x
        flat = rng.choice(n * p.geom.n_y, 256, replace=False)       # distinct pixels
        pix = np.stack([flat % n, flat // n], 1).astype(np.int32)
        hkl = oracle_hkl(orc, p, s.hkl_host)
        M = orc.intensities_M(p, hkl)
        I, E = orc.pattern(p, hkl, M, pix)
        # targets off the model by up to 0.3 max I everywhere, so every residual
        # is large against the image gate (1e-5 max I)
        It = np.maximum(I + 0.3 * I.max() * rng.uniform(-1.0, 1.0, len(I)), 0.0)
        It = It.astype(np.float32).astype(np.float64)
        t = np.zeros((p.geom.n_y, n), np.float32)
        m = np.zeros((p.geom.n_y, n), np.float32)
        t[pix[:, 1], pix[:, 0]] = It
        m[pix[:, 1], pix[:, 0]] = 1.0
        pixes.append(pix), Io.append(I), Eo.append(E), Its.append(It)
        targets.append(torch.as_tensor(t, device="cuda")), masks.append(torch.as_tensor(m, device="cuda"))
    step = gpu.BatchStep([s.prob for s in sims], [s.atoms for s in sims], targets=targets, masks=masks)
    step()
    torch.cuda.synchronize()
    for k, (p, s) in enumerate(zip(models, sims)):
        pix = pixes[k]
        got = step.images[k].cpu().numpy()[pix[:, 1], pix[:, 0]]
        assert Io[k].max() > 0, chosen[k]
        mr, l2 = parity(got, Io[k])
        assert mr <= MAX_REL and l2 <= L2_REL, (chosen[k], mr, l2)
        cnt = s.evals()
        torch.cuda.synchronize()
        c = cnt.cpu().numpy()[pix[:, 1], pix[:, 0]]
        assert np.all(c >= Eo[k][:, 1]) and np.all(c <= Eo[k][:, 2]), chosen[k]
        loss_o, go, _ = orc.full_gradient(p, oracle_hkl(orc, p, s.hkl_host), Its[k], pix)
        # the loss bound that follows from the image gate: |I - I_o| <= d =
        # MAX_REL max I_o per pixel gives |dL| <= sum w (2 |I_o - I_t| d + d^2)
        d = MAX_REL * Io[k].max()
        w = 1.0 / (Its[k] + 1.0)
        bound = float(np.sum(w * (2.0 * np.abs(Io[k] - Its[k]) * d + d * d)))
        assert abs(step.losses[k].item() - loss_o) <= bound, (chosen[k], step.losses[k].item(), loss_o, bound)
        for got_t, ref, what in ((step.dfrac[k], go["frac"], "frac"), (step.dB[k], go["B"], "B")):
            got_a = got_t.cpu().numpy().reshape(-1)
            ref_a = np.asarray(ref, np.float64).reshape(-1)
            scale = np.max(np.abs(ref_a))
            assert scale > 0, (chosen[k], what)
            err = np.max(np.abs(got_a - ref_a)) / scale
            l2 = np.linalg.norm(got_a - ref_a) / np.linalg.norm(ref_a)
            assert err <= ADJ_TOL and l2 <= ADJ_TOL, (chosen[k], what, err, l2)
        dg = step.dglobal[k].cpu().numpy()
        ref_g = np.concatenate([go["L"], go["g"], [go["sigma"], go["gamma"]]])
        for i, name in enumerate(["dL_a", "dL_b", "dL_c", "dg_a", "dg_b", "dg_c", "dsigma", "dgamma"]):
            if ref_g[i] == 0.0:
                assert abs(dg[i]) <= 1e-6 * np.max(np.abs(ref_g)), (chosen[k], name)
            else:
                assert dg[i] == pytest.approx(ref_g[i], rel=ADJ_TOL), (chosen[k], name, dg[i], ref_g[i])


def test_large_structure_factors(gpu, orc):
    """Structure factors of the large workload against the oracle: every
    meridional reflection (h = k = 0, where consecutive-l groups would
    multiply factors of the same angle, whose errors would then add up instead
    of averaging out: 5e-6 of the amplitude scale for (0, 0, 2) before such
    reflections were evaluated directly) to 1e-6 of the amplitude scale
    sqrt(sum amp^2), a seeded 8,000-reflection sample to the general
    structure-factor tolerance, and M consistent with F's error."""
    import torch
    from _common import SF_TOL, amp_scale
    p = api_precision(W.config2(0.01))
    sim = gpu.Simulation(p)
    F, M = sim.structure_factors()
    torch.cuda.synchronize()
    h = oracle_hkl(orc, p, sim.hkl_host)
    mer = np.where((h[:, 0] == 0) & (h[:, 1] == 0))[0]
    rng = np.random.default_rng(8000)
    idx = np.unique(np.concatenate([mer, rng.choice(len(h), 8000, replace=False)]))
    Fo = orc.structure_factors(p.cell, p.atoms, h[idx])
    Mo = orc.intensities_M(p, h[idx], Fo)
    Fg = F.cpu().numpy()[idx].astype(np.float64)
    Mg = M.cpu().numpy()[idx].astype(np.float64)
    scale = amp_scale(p, h[idx])
    err = np.abs((Fg[:, 0] + 1j * Fg[:, 1]) - Fo) / scale
    is_mer = np.isin(idx, mer)
    assert is_mer.sum() >= 80 and err[is_mer].max() <= 1e-6, (err[is_mer].max(), h[idx][is_mer][np.argmax(err[is_mer])])
    assert err.max() <= SF_TOL, (err.max(), h[idx][np.argmax(err)])
    d = SF_TOL * scale
    pdw = Mo / np.maximum(np.abs(Fo) ** 2, 1e-300)
    assert np.all(np.abs(Mg - Mo) <= (2.0 * np.abs(Fo) + d) * d * pdw + 1e-6 * Mo)
