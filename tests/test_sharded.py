"""Reflection-sharded refinement step (paper_2608_23245_b300/sharded.py).

CPU, gloo, world size 2 and 3: ranks own contiguous slices of the reflection
list, compute their slice's partial image and partial gradients, and the step
exchanges them by all-reduce.  The slice computations here are the FP64
oracle's (a stand-in backend: the exchange logic is what is under test), so
the sharded result must equal the one-rank result to rounding (1e-12
relative): the image and every gradient are sums over reflections.

GPU (one device): the library backend's slices, evaluated one after another
and summed, against the unsharded library calls."""
import os
import socket

import numpy as np
import pytest
import torch

from paper_2608_23245_b300 import sharded, workloads as W
from _common import api_precision


def _tiny():
    from dataclasses import replace
    p = W.small_triclinic()
    br = replace(p.br, n_nodes=10)
    geom = replace(p.geom, n_x=30, n_y=22, pixel=1.2)
    atoms = W.Atoms(frac=p.atoms.frac[:12].copy(), B=p.atoms.B[:12].copy(), occ=p.atoms.occ[:12].copy(),
                    elem=p.atoms.elem[:12].copy(), ff=8000.0 * p.atoms.ff)
    return replace(p, br=br, geom=geom, atoms=atoms, d_min=4.0)


class OracleBackend:
    """The slice computations by the FP64 oracle (tests only)."""

    def __init__(self, problem, target):
        import oracle
        oracle.build()
        self.o = oracle
        self.p = problem
        self.hkl = oracle.reflections(problem.cell, problem.d_min, problem.d_max)
        self.F = oracle.structure_factors(problem.cell, problem.atoms, self.hkl)
        _, self.P, self.DW = oracle.refl_scalars(problem, self.hkl)
        self.F2 = np.abs(self.F) ** 2
        self.M = self.F2 * self.P * self.DW
        self.target = target

    def partial_image(self, b, e):
        I, _ = self.o.pattern(self.p, self.hkl[b:e], self.M[b:e])
        return torch.as_tensor(I, dtype=torch.float64)

    def loss_grad(self, image):
        loss, gI = self.o.loss_and_grad(image.numpy(), self.target)
        return loss, gI

    def partial_grads(self, b, e, gI):
        G, dbeta, ds, dg = self.o.pattern_adjoint(self.p, self.hkl[b:e], self.M[b:e], gI)
        dL, dgg = self.o.chain_globals(self.p, self.hkl[b:e], self.F2[b:e], G, dbeta)
        dfrac, dB = self.o.sf_adjoint(self.p.cell, self.p.atoms, self.hkl[b:e], self.F[b:e],
                                      G * self.P[b:e] * self.DW[b:e])
        glob = np.concatenate([dL, dgg, [ds, dg]])
        return torch.as_tensor(dfrac), torch.as_tensor(dB), torch.as_tensor(glob)

    @staticmethod
    def pack(dfrac, dB, dglob):
        return torch.cat([dfrac.reshape(-1), dB.reshape(-1), dglob.reshape(-1)])

    @staticmethod
    def unpack(packed, dfrac, dB, dglob):
        n3, n1 = dfrac.numel(), dB.numel()
        return (packed[:n3].reshape(dfrac.shape), packed[n3:n3 + n1].reshape(dB.shape),
                packed[n3 + n1:].reshape(dglob.shape))


def _target(p):
    rng = np.random.default_rng(77)
    return rng.uniform(0.0, 2.0, p.geom.n_x * p.geom.n_y)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_2608_23245_b300 import replicas
    replicas.dist_init("gloo")
    p = _tiny()
    be = OracleBackend(p, _target(p))
    step = sharded.ShardedRefineStep(be, len(be.hkl), rank, world)
    img, loss, dfrac, dB, dglob = step()
    out.put((rank, step.begin, step.end, img.numpy(), loss, dfrac.numpy(), dB.numpy(), dglob.numpy()))
    dist.destroy_process_group()


def _run(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    return res


def _rel(a, b):
    a, b = np.asarray(a, np.float64).reshape(-1), np.asarray(b, np.float64).reshape(-1)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_sharded_step_equals_one_rank(world):
    p = _tiny()
    be = OracleBackend(p, _target(p))
    n = len(be.hkl)
    img1, loss1, dfrac1, dB1, dglob1 = sharded.ShardedRefineStep(be, n, 0, 1)()
    assert float(img1.max()) > 0 and n >= 3 * world
    res = _run(world)
    spans = [(r[1], r[2]) for r in res]
    assert spans[0][0] == 0 and spans[-1][1] == n and all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
    for r in res:
        assert _rel(r[3], img1.numpy()) <= 1e-12
        assert r[4] == pytest.approx(loss1, rel=1e-12)
        assert _rel(r[5], dfrac1.numpy()) <= 1e-12
        assert _rel(r[6], dB1.numpy()) <= 1e-12
        assert _rel(r[7], dglob1.numpy()) <= 1e-12


def test_slices_partition():
    for n, world in ((0, 2), (5, 8), (217252, 8), (100, 3)):
        spans = [sharded.reflection_slice(n, r, world) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))


@pytest.mark.gpu
def test_library_slices_sum_to_unsharded_step():
    """On one GPU: the library backend over three reflection slices, run one
    after another and summed (what the all-reduces do across GPUs), against
    the unsharded forward and adjoint of the same model."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2608_23245_b300 import _build, fdx
    _build.build()
    p = api_precision(W.small_helix())
    sim = fdx.Simulation(p)
    img_ref = sim.forward().clone()
    target = (img_ref * 0.8 + 0.01).contiguous()
    gI = torch.empty_like(img_ref)
    loss_ref, _ = fdx.fdx_loss(img_ref, target, None, dL_dI=gI)
    na = p.atoms.n
    ref = [torch.empty((na, 3), dtype=torch.float64, device="cuda"), torch.empty(na, dtype=torch.float64, device="cuda"),
           torch.empty(8, dtype=torch.float64, device="cuda")]
    fdx.fdx_pattern_backward(sim.prob, sim.atoms, sim.F, gI, *ref)
    be = sharded.FdxBackend(p, target)
    n = be.hkl.shape[0]
    world = 3
    spans = [sharded.reflection_slice(n, r, world) for r in range(world)]
    img = torch.zeros_like(img_ref)
    for b, e in spans:
        img += be.partial_image(b, e)
    loss, gI2 = be.loss_grad(img)
    sums = [torch.zeros_like(t) for t in ref]
    for b, e in spans:
        for acc, part in zip(sums, be.partial_grads(b, e, gI2)):
            acc += part
    torch.cuda.synchronize()
    assert _rel(img.cpu().numpy(), img_ref.cpu().numpy()) <= 1e-6
    assert loss.item() == pytest.approx(loss_ref.item(), rel=1e-5)
    for got, want in zip(sums, ref):
        assert _rel(got.cpu().numpy(), want.cpu().numpy()) <= 1e-5


@pytest.mark.gpu
def test_nccl_all_reduce_path_one_rank():
    """The sharded step's exchanges through NCCL on CUDA tensors (a one-rank
    process group on this GPU: every all-reduce is the identity, so the step
    must equal the same step with no exchange bit for bit).  Runs in a child
    process so that the process group does not outlive the test."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    pr = ctx.Process(target=_nccl_worker, args=(_free_port(), q))
    pr.start()
    ok, msg = q.get(timeout=300)
    pr.join(timeout=60)
    assert pr.exitcode == 0 and ok, msg


def _nccl_worker(port, q):
    try:
        import os
        import torch.distributed as dist
        os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
        os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
        torch.cuda.set_device(0)
        dist.init_process_group("nccl", rank=0, world_size=1)
        from paper_2608_23245_b300 import _build
        _build.build()
        p = api_precision(W.small_helix())
        be = sharded.FdxBackend(p, None)
        img0 = be.partial_image(0, be.hkl.shape[0]).clone()
        target = (img0 * 0.8 + 0.01).contiguous()
        be = sharded.FdxBackend(p, target)
        n = be.hkl.shape[0]
        # the backend returns its own buffers: keep copies of the first step's results
        plain = [x.clone() if torch.is_tensor(x) else x for x in sharded.ShardedRefineStep(be, n, 0, 1)()]
        viaccl = sharded.ShardedRefineStep(be, n, 0, 1, reduce=sharded._all_reduce_sum)()
        torch.cuda.synchronize()
        same = all(torch.equal(a, b) if torch.is_tensor(a) else a == b for a, b in zip(plain, viaccl))
        dist.destroy_process_group()
        q.put((bool(same) and float(plain[0].max()) > 0, "nccl step differs" if not same else ""))
    except Exception as e:  # report to the parent instead of hanging it
        q.put((False, repr(e)))
