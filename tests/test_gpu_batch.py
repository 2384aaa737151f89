"""Batched refinement (fdx_batch_refine): one step for several models with
the pattern of all models in one persistent launch and the adjoint of all
models in another.  The batched step must give the same images, losses and
gradients as the per-model entry points (same kernels per item: bitwise), the
per-model forward must agree with the FP64 oracle, and a CUDA-graph replay of
the batched step must reproduce the eager step exactly."""
import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W
from _common import L2_REL, MAX_REL, api_precision, oracle_hkl, parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2608_23245_b300 import _build, fdx
    _build.build()
    return fdx


def _setup(gpu, n=5):
    import torch
    models = [api_precision(p) for p in W.small_batch(n)]
    targets = [api_precision(W.config4_target(p, m)) for m, p in enumerate(models)]
    sims = [gpu.Simulation(p) for p in models]
    tims = [gpu.Simulation(t).forward().clone() for t in targets]
    probs = [s.prob for s in sims]
    return models, sims, tims, probs


def _per_model(gpu, sims, tims):
    import torch
    out = []
    for s, It in zip(sims, tims):
        s.forward()
        gI = torch.empty_like(s.image)
        loss, _ = gpu.fdx_loss(s.image, It, None, dL_dI=gI)
        na = s.atoms.frac.shape[0]
        dfrac = torch.empty((na, 3), dtype=torch.float64, device="cuda")
        dB = torch.empty(na, dtype=torch.float64, device="cuda")
        dg = torch.empty(8, dtype=torch.float64, device="cuda")
        dM = torch.empty(s.hkl.shape[0], dtype=torch.float32, device="cuda")
        gpu.fdx_pattern_backward(s.prob, s.atoms, s.F, gI, dfrac, dB, dg, dM)
        out.append(dict(image=s.image.clone(), F=s.F.clone(), loss=loss.clone(), dfrac=dfrac, dB=dB, dg=dg, dM=dM))
    torch.cuda.synchronize()
    return out


def test_batch_matches_per_model(gpu):
    import torch
    models, sims, tims, probs = _setup(gpu)
    ref = _per_model(gpu, sims, tims)
    step = gpu.BatchStep(probs, [s.atoms for s in sims], targets=tims)
    step()
    torch.cuda.synchronize()
    for m in range(len(models)):
        assert torch.equal(step.images[m], ref[m]["image"]), m
        assert torch.equal(step.F[m], ref[m]["F"]), m
        assert step.losses[m].item() == ref[m]["loss"].item(), m
        assert torch.equal(step.dfrac[m], ref[m]["dfrac"]), m
        assert torch.equal(step.dB[m], ref[m]["dB"]), m
        assert torch.equal(step.dglobal[m], ref[m]["dg"]), m
        assert torch.equal(step.dM[m][:ref[m]["dM"].shape[0]], ref[m]["dM"]), m
        assert float(step.images[m].max()) > 0


def test_batch_forward_against_oracle(gpu, orc):
    import torch
    models, sims, tims, probs = _setup(gpu, 3)
    step = gpu.BatchStep(probs, [s.atoms for s in sims])
    step()
    torch.cuda.synchronize()
    for m, p in enumerate(models):
        hkl = oracle_hkl(orc, p, sims[m].hkl_host)
        I, _ = orc.pattern(p, hkl, orc.intensities_M(p, hkl))
        mr, l2 = parity(step.images[m].cpu().numpy().reshape(-1), I)
        assert mr <= MAX_REL and l2 <= L2_REL, (m, mr, l2)


def test_batch_graph_replay(gpu):
    """The whole batched step captured in a CUDA graph and replayed twice,
    with the atoms' coordinates changed in place between replays."""
    import torch
    models, sims, tims, probs = _setup(gpu, 4)
    step = gpu.BatchStep(probs, [s.atoms for s in sims], targets=tims)
    step()
    torch.cuda.synchronize()
    eager_img = [x.clone() for x in step.images]
    eager_df = [x.clone() for x in step.dfrac]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        step(s)  # warm-up on the capture stream
        torch.cuda.current_stream().synchronize()
        with torch.cuda.graph(g, stream=s):
            step(s)
    torch.cuda.current_stream().wait_stream(s)
    for x in step.images:
        x.zero_()
    g.replay()
    torch.cuda.synchronize()
    for m in range(len(models)):
        assert torch.equal(step.images[m], eager_img[m]), m
        assert torch.equal(step.dfrac[m], eager_df[m]), m
    # move the atoms of model 0 (device memory read by the graph) and replay
    sims[0].atoms.frac.add_(1e-3)
    g.replay()
    torch.cuda.synchronize()
    assert not torch.equal(step.images[0], eager_img[0])
    ref = _per_model(gpu, sims[:1], tims[:1])
    assert torch.equal(step.images[0], ref[0]["image"])
    assert torch.equal(step.dfrac[0], ref[0]["dfrac"])


def test_batch_mixed_tile_shapes(gpu):
    """Models of both tile shapes in one batch (the reduced models take one
    pixel per lane; the helix with 0.2 mm pixels two): one persistent launch
    per shape and kernel, each model still bitwise equal to its per-model
    entry points."""
    import torch
    from dataclasses import replace
    h = W.small_helix()
    fine = replace(h, geom=replace(h.geom, pixel=0.2))
    models = [api_precision(p) for p in W.small_batch(2)] + [api_precision(fine)] + \
             [api_precision(W.small_batch(3)[2])]
    targets = [api_precision(W.config4_target(p, m)) if m != 2 else api_precision(replace(
        p, br=replace(p.br, g=(0.025, 0.025, 0.0)))) for m, p in enumerate(models)]
    sims = [gpu.Simulation(p) for p in models]
    tims = [gpu.Simulation(t).forward().clone() for t in targets]
    probs = [s.prob for s in sims]
    ref = _per_model(gpu, sims, tims)
    step = gpu.BatchStep(probs, [s.atoms for s in sims], targets=tims)
    step()
    torch.cuda.synchronize()
    for m in range(len(models)):
        assert torch.equal(step.images[m], ref[m]["image"]), m
        assert step.losses[m].item() == ref[m]["loss"].item(), m
        assert torch.equal(step.dfrac[m], ref[m]["dfrac"]), m
        assert torch.equal(step.dB[m], ref[m]["dB"]), m
        assert torch.equal(step.dglobal[m], ref[m]["dg"]), m
        assert float(step.images[m].max()) > 0
