"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: density fields, neutral fractions, source
catalogues, ensemble layouts and loss weights.  It holds none of the ray
tracing or chemistry arithmetic, so both the CUDA library's tests/benchmark
and the CPU oracle can consume the same inputs.

The paper's cosmological inputs (N-body density and halo catalogues of a
349 Mpc box, Sec. 5) are not available; these generators stand in for them:

* density: lognormal field n_H = nbar exp(sigma g - sigma^2/2) from a Gaussian
  random field g with power spectrum P(k) ~ k^-2 (k = 0 mode removed, unit
  sample variance), rescaled so that the sample mean is exactly nbar;
* x_HI: i.i.d. uniform on [0, 1);
* sources: the n_src densest cells (ties broken by linear index), photon rates
  log-uniform, radius either fixed or R = 5 (Ndot/1e50)^(1/5) cells (5..50 for
  Ndot in [1e50, 1e55]).

Seeds follow one base seed 2311_01492: field +0, x_HI +1, sources +2,
ensemble layout +3, loss weights +4.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as _fft

MPC_CM = 3.0856775814913673e24
KPC_CM = 3.0856775814913673e21
MYR_S = 3.15576e13
BASE_SEED = 2311_01492


def lognormal_field(n, mean, sigma_ln=1.0, slope=-2.0, seed=BASE_SEED):
    """FP64 lognormal field on an n^3 periodic grid, C order, sample mean == mean."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    workers = max(1, len(os.sched_getaffinity(0)))
    F = _fft.rfftn(white, workers=workers)
    del white
    k1 = np.fft.fftfreq(n) * n
    k3 = np.fft.rfftfreq(n) * n
    k2 = k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + k3[None, None, :] ** 2
    with np.errstate(divide="ignore"):
        amp = np.where(k2 > 0, k2 ** (slope / 4.0), 0.0)  # sqrt(P(k)), P ~ k^slope
    F *= amp
    g = _fft.irfftn(F, s=(n, n, n), axes=(0, 1, 2), workers=workers)
    g /= g.std()
    f = mean * np.exp(sigma_ln * g - 0.5 * sigma_ln ** 2)
    f *= mean / f.mean()
    return np.ascontiguousarray(f, dtype=np.float64)


def uniform_xhi(n, seed=BASE_SEED + 1):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(n, n, n))


def densest_cells(field, nsrc):
    """(nsrc, 3) int32 positions of the nsrc largest values (ties: lower linear index first)."""
    n = field.shape[0]
    flat = field.reshape(-1)
    nsrc = min(nsrc, flat.size)
    if nsrc < flat.size:
        cand = np.argpartition(-flat, nsrc - 1)[:nsrc]
    else:
        cand = np.arange(flat.size)
    order = np.lexsort((cand, -flat[cand]))
    idx = cand[order]
    return np.stack(np.unravel_index(idx, (n, n, n)), axis=1).astype(np.int32)


def loguniform(lo, hi, size, rng):
    return 10.0 ** rng.uniform(np.log10(lo), np.log10(hi), size=size)


def radius_from_ndot(ndot):
    """R = 5 (Ndot/1e50)^(1/5) cells: 5..50 for Ndot in [1e50, 1e55]."""
    return 5.0 * (np.asarray(ndot) / 1e50) ** 0.2


def catalogue(nH, nsrc, ndot_lo, ndot_hi, radius=None, seed=BASE_SEED + 2):
    rng = np.random.default_rng(seed)
    pos = densest_cells(nH, nsrc)
    ndot = loguniform(ndot_lo, ndot_hi, pos.shape[0], rng)
    if radius is None:
        R = radius_from_ndot(ndot)
    else:
        R = np.full(pos.shape[0], float(radius))
    return pos, ndot, R


def loss_weights(shape, seed=BASE_SEED + 4):
    return np.random.default_rng(seed).standard_normal(shape)


# --------------------------------------------------------------------------
# Workloads (grid, box, field recipe, catalogue), named by what they are.

def single_source_uniform(n=32, box_mpc=10.0, nH=1e-3, xhi=1.0, ndot=1e54, radius=16.0):
    """One source at the centre of a uniform, fully neutral box (closed-form checks)."""
    c = n // 2
    return dict(n=n, cell_cm=box_mpc * MPC_CM / n,
                nH=np.full((n, n, n), nH), xHI=np.full((n, n, n), xhi),
                pos=np.array([[c, c, c]], dtype=np.int32), ndot=np.array([ndot]),
                radius=np.array([radius]), spectrum="bb", T_bb=5e4)


def lognormal_box(n, box_mpc, nsrc, ndot_lo, ndot_hi, radius=None, mean=2e-4, sigma_ln=1.0,
                  seed=BASE_SEED):
    """Lognormal P(k)~k^-2 density, uniform x_HI, sources at the densest cells."""
    nH = lognormal_field(n, mean, sigma_ln, seed=seed)
    xHI = uniform_xhi(n, seed=seed + 1)
    pos, ndot, R = catalogue(nH, nsrc, ndot_lo, ndot_hi, radius, seed=seed + 2)
    return dict(n=n, cell_cm=box_mpc * MPC_CM / n, nH=nH, xHI=xHI, pos=pos, ndot=ndot,
                radius=R, spectrum="bb", T_bb=5e4)


def box128_1e4():
    """128^3, 100 Mpc, 1e4 sources, Ndot log-U[1e50,1e54], R = 32."""
    return lognormal_box(128, 100.0, 10_000, 1e50, 1e54, radius=32.0)


def box250_1e6(nsrc=1_000_000):
    """250^3, 349 Mpc, ~1e6 sources, Ndot log-U[1e50,1e55], R = 5..50 by luminosity."""
    return lognormal_box(250, 349.0, nsrc, 1e50, 1e55, radius=None)


def ensemble_layout(nbox=64, sizes=(32, 48, 64, 96, 128), nsrc_lo=10, nsrc_hi=5000,
                    seed=BASE_SEED + 3):
    """Grid size and source count of each box of an ensemble."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=nbox)
    cnt = np.floor(loguniform(nsrc_lo, nsrc_hi + 1, nbox, rng)).astype(int)
    cnt = np.clip(cnt, nsrc_lo, nsrc_hi)
    return ns, cnt


def ensemble(nbox=64, cell_mpc=0.78125, seed=BASE_SEED, **kw):
    """Boxes with the lognormal recipe; R = 5..50 by luminosity, clipped to the window."""
    ns, cnt = ensemble_layout(nbox, seed=seed + 3, **kw)
    boxes = []
    for b, (n, c) in enumerate(zip(ns, cnt)):
        bs = seed + 1000 * (b + 1)
        nH = lognormal_field(int(n), 2e-4, 1.0, seed=bs)
        xHI = uniform_xhi(int(n), seed=bs + 1)
        pos, ndot, R = catalogue(nH, int(c), 1e50, 1e55, None, seed=bs + 2)
        R = np.minimum(R, n // 2)
        boxes.append(dict(n=int(n), cell_cm=cell_mpc * MPC_CM, nH=nH, xHI=xHI, pos=pos,
                          ndot=ndot, radius=R))
    return boxes
