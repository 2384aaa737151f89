"""The library built with its bounds checks (FDX_DEBUG, libfdx_debug.so) run
over every entry point on workloads that reach the edge cases -- ragged
detectors, node grids of 1 to 512 per axis, both tile shapes, two element
passes of the structure factors, every lineshape, the adjoint, the scatter
form with detector spots, the ring average, a batch of mixed tile shapes and
the allocation-free structure factors -- must record no out-of-bounds index
(fdx_debug_status; a deliberate failure from fdx_debug_probe shows that
failures are recorded), and its image must still match the oracle.  It runs
in a process of its own (one library per process)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _debug_worker(q):
    try:
        import os
        import sys
        from dataclasses import replace
        here = os.path.dirname(os.path.abspath(__file__))
        sys.path.insert(0, here)
        sys.path.insert(0, os.path.dirname(here))
        import torch
        from paper_2608_23245_b300 import _build, fdx, workloads as W
        from _common import api_precision
        fdx.LIB_PATH = _build.build(debug=True)
        assert fdx.fdx_debug_status()[0], "the debug build has no checks compiled in"
        # the recording itself: one deliberate failure is reported, then cleared
        assert fdx.fdx_debug_probe()
        torch.cuda.synchronize()
        assert fdx.fdx_debug_status() == (True, 1 << 63, 7)
        assert fdx.fdx_debug_status() == (True, 0, 0)
        out = {}
        h = api_precision(W.small_helix())
        fine = replace(h, geom=replace(h.geom, pixel=0.2))
        for name, p in (("helix", h), ("fine", fine), ("sinc", api_precision(W.small_sinc())),
                        ("gauss", api_precision(W.small_gauss())), ("tilted", api_precision(W.small_tilted())),
                        ("config0", api_precision(W.config0()))):
            sim = fdx.Simulation(p)
            img = sim.forward()
            sim.evals()
            if name in ("helix", "fine", "sinc"):
                gI = torch.ones_like(img) * 1e-3
                n, na = sim.hkl.shape[0], p.atoms.n
                g = [torch.empty((na, 3), dtype=torch.float64, device="cuda"),
                     torch.empty(na, dtype=torch.float64, device="cuda"),
                     torch.empty(8, dtype=torch.float64, device="cuda"),
                     torch.empty(n, dtype=torch.float32, device="cuda")]
                fdx.fdx_pattern_backward(sim.prob, sim.atoms, sim.F, gI, *g)
            if name == "helix":
                out["helix_image"] = img.cpu().numpy()
                out["helix_hkl"] = sim.hkl_host
                samples = torch.as_tensor(W.scatter_samples(4, 8, 8), device="cuda")
                sim.scatter(samples, spot_size=3)
                sim.ring()
        for nn in (1, 130, 512):
            p = replace(h, br=replace(h.br, n_nodes=nn), geom=replace(h.geom, n_x=17, n_y=13))
            fdx.Simulation(p).forward()
        # two element passes of the structure factors (48 types)
        a = h.atoms
        ff = np.tile(a.ff, (12, 1))[:48]
        many = replace(h, atoms=replace(a, elem=(np.arange(a.n) % 48).astype(np.uint8), ff=ff))
        fdx.Simulation(many).structure_factors()
        # batch of both tile shapes, with the loss and the adjoint
        models = [api_precision(m) for m in W.small_batch(2)] + [fine]
        sims = [fdx.Simulation(m) for m in models]
        tims = [s.forward().clone() * 1.1 for s in sims]
        fdx.BatchStep([s.prob for s in sims], [s.atoms for s in sims], targets=tims)()
        # allocation-free structure factors
        sim = fdx.Simulation(h)
        fdx.fdx_structure_factors_noalloc(h.cell, sim.atoms, sim.hkl, h.br)
        torch.cuda.synchronize()
        enabled, flags, index = fdx.fdx_debug_status()
        out.update(enabled=enabled, flags=flags, index=index)
        q.put((True, out))
    except Exception as e:  # report to the parent instead of hanging it
        import traceback
        q.put((False, traceback.format_exc()))


def test_debug_build_records_no_out_of_bounds_index(orc):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    pr = ctx.Process(target=_debug_worker, args=(q,))
    pr.start()
    ok, out = q.get(timeout=1200)
    pr.join(timeout=120)
    assert ok, out
    assert pr.exitcode == 0
    assert out["enabled"]
    assert out["flags"] == 0, "failed checks 0x%x, last index %d" % (out["flags"], out["index"])
    from paper_2608_23245_b300 import workloads as W
    from _common import L2_REL, MAX_REL, api_precision, oracle_hkl, parity
    p = api_precision(W.small_helix())
    hkl = oracle_hkl(orc, p, out["helix_hkl"])
    I, _ = orc.pattern(p, hkl, orc.intensities_M(p, hkl))
    mr, l2 = parity(out["helix_image"].reshape(-1), I)
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)
