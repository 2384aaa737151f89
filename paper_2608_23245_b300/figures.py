"""The paper's two model figures with |F| = 1, computed through the GPU path.

Fig. GvL compares a Gaussian (sigma = 3 deg) and a Lorentzian (gamma = 3 deg)
crystal orientation distribution on the same lattice; Fig. equator shows the
intensity profile along the equator for several isotropic disorder
parameters (paracrystal g, axis Debye-Waller B).  Both use the hexagonal model
cell a = b = 10 A, c = 5 A, gamma = 120 deg and F_hkl = 1 (one atom at the
origin with f = 1, B = 0; inputs in ``workloads.gvl`` / ``workloads.equator``).

Everything here runs on the GPU through the library (structure factors, then
the gather-form pattern); this module only selects rows and writes files.

    python -m paper_2608_23245_b300.figures --out DIR [--gvl-px 511] [--equator-px 1023]

writes ``gvl_gauss.npy``, ``gvl_lorentz.npy`` (float32 images, row j along
+fiber) with log-scaled ``.pgm`` views, and ``equator.npz`` (one profile per
(g, B), with the pixel centres' distance from the beam centre in mm).
"""
from __future__ import annotations

import argparse
import os
from typing import Dict, Iterable, Tuple

import numpy as np

from . import workloads as W

EQUATOR_PARAMS = ((0.0, 0.0), (0.01, 0.0), (0.03, 0.0), (0.05, 0.0), (0.03, 10.0))


def simulate(problem) -> np.ndarray:
    """Structure factors and pattern of one problem on the GPU; the image as a
    host float32 array [n_y][n_x]."""
    import torch
    from . import fdx
    sim = fdx.Simulation(problem)
    img = sim.forward()
    torch.cuda.synchronize()
    return img.cpu().numpy()


def gvl_images(n_px: int = 511, n_nodes: int = 64) -> Dict[str, np.ndarray]:
    """Fig. GvL: the two detector images, keyed 'gauss' and 'lorentz'."""
    return {k: simulate(W.gvl(k, n_px=n_px, n_nodes=n_nodes)) for k in ("gauss", "lorentz")}


def equator_row(image: np.ndarray) -> np.ndarray:
    """The detector row on the equator (the middle row of an odd-height
    image: its pixel centres have Z = 0)."""
    n_y = image.shape[0]
    if n_y % 2 == 0:
        raise ValueError("the equator lies between two rows of an even-height image")
    return image[n_y // 2]


def equator_profiles(params: Iterable[Tuple[float, float]] = EQUATOR_PARAMS, n_x: int = 1023, n_y: int = 15,
                     n_nodes: int = 48) -> Tuple[np.ndarray, Dict[Tuple[float, float], np.ndarray]]:
    """Fig. equator: for each (g, B) the equatorial row of the strip detector,
    and the pixel centres' horizontal distance from the beam centre (mm)."""
    out = {}
    x_mm = None
    for g, B in params:
        p = W.equator(g, B, n_x=n_x, n_y=n_y, n_nodes=n_nodes)
        out[(g, B)] = equator_row(simulate(p))
        x_mm = (np.arange(n_x) + 0.5 - 0.5 * n_x) * p.geom.pixel
    return x_mm, out


def write_pgm(path: str, image: np.ndarray, decades: float = 4.0) -> None:
    """An 8-bit binary PGM of log10(image / max) over the top `decades`, row 0
    at the top (the image's last row, +fiber), for viewing without a plotting
    library."""
    img = np.asarray(image, dtype=np.float64)
    mx = float(img.max()) if img.size else 0.0
    if mx > 0:
        x = np.log10(np.maximum(img / mx, 10.0 ** -decades)) / decades + 1.0
    else:
        x = np.zeros_like(img)
    g = np.clip(np.rint(255.0 * x), 0, 255).astype(np.uint8)[::-1]
    with open(path, "wb") as f:
        f.write(b"P5\n%d %d\n255\n" % (g.shape[1], g.shape[0]))
        f.write(np.ascontiguousarray(g).tobytes())


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--gvl-px", type=int, default=511)
    ap.add_argument("--equator-px", type=int, default=1023)
    a = ap.parse_args(argv)
    os.makedirs(a.out, exist_ok=True)
    for k, img in gvl_images(a.gvl_px).items():
        np.save(os.path.join(a.out, "gvl_%s.npy" % k), img)
        write_pgm(os.path.join(a.out, "gvl_%s.pgm" % k), img)
    x_mm, prof = equator_profiles(n_x=a.equator_px)
    keys = sorted(prof)
    np.savez(os.path.join(a.out, "equator.npz"), x_mm=x_mm, g=np.array([k[0] for k in keys]),
             B=np.array([k[1] for k in keys]), profiles=np.stack([prof[k] for k in keys]))


if __name__ == "__main__":
    main()
