"""Adjoint (rt_raytrace_backward) against the oracle's complex-step derivatives,
the linearity closed form in Ndot, and central finite differences of the GPU
forward.  L = sum_p w_p Gamma_p."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2311_01492_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2311_01492_gb300 import build
    build.build()


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dtype).contiguous()


def gpu_grid(n, cell, nH, xHI, pos, ndot, R, tab):
    from paper_2311_01492_gb300 import api
    g = api.Grid(n, cell)
    if tab.kind == 1:
        g.set_tables("grey_exact")
    else:
        g.set_tables("knots", g=tab.g, h=tab.h)
    g.set_density(dev(nH))
    g.set_xHI(dev(xHI))
    g.set_sources(dev(pos, torch.int32), dev(ndot), dev(R))
    return g


def _box(n, seed, xhi_scale, nsrc):
    rng = np.random.default_rng(seed)
    nH = S.lognormal_field(n, 1e-3, sigma_ln=0.6, seed=seed).reshape(-1)
    xHI = (xhi_scale * rng.uniform(0.2, 1.0, n ** 3))
    pos = rng.integers(0, n, (nsrc, 3)).astype(np.int32)
    ndot = 10 ** rng.uniform(49, 51, nsrc)
    R = rng.uniform(3.0, n / 2.0 + 2.0, nsrc)
    w = S.loss_weights(n ** 3, seed=seed + 4)
    return nH, xHI, pos, ndot, R, w


@pytest.mark.parametrize("spec,xhi_scale,stop", [("grey_exact", 3e-3, True), ("bb", 3e-3, True),
                                                  ("bb", 1e-9, True), ("bb", 0.3, True),
                                                  ("bb", 0.3, False), ("grey_exact", 0.3, True)])
def test_adjoint_matches_oracle_complex_step(spec, xhi_scale, stop):
    n = 12
    cell = 10 * S.KPC_CM
    nH, xHI, pos, ndot, R, w = _box(n, 41, xhi_scale, 4)
    tab = O.make_table(spec)
    g = gpu_grid(n, cell, nH, xHI, pos, ndot, R, tab)
    g.set_adjoint_mode(stop)
    dn, dq = g.backward(dev(w))
    dn = dn.cpu().numpy()
    dq = dq.cpu().numpy()
    g.stats()
    cells = np.arange(n ** 3, dtype=np.int64)
    dn_o, dq_o = O.loss_grad_cs(n, cell, nH, xHI, pos, ndot, R, tab, w, cells, np.arange(len(ndot)),
                                nthreads=8)
    scale = np.abs(dn_o).max()
    assert scale > 0
    assert np.linalg.norm(dn - dn_o) <= 1e-9 * np.linalg.norm(dn_o)
    if xhi_scale < 1e-6:
        # dtau ~ tau_lim: Gamma barely depends on n_HI, so dL/dlog n_HI is the
        # near-cancellation of -w Gamma and dtau ds lambda; both sides lose
        # ~eps/dtau relative to those terms.
        np.testing.assert_allclose(dn, dn_o, rtol=1e-6, atol=1e-12 * scale)
    else:
        np.testing.assert_allclose(dn, dn_o, rtol=1e-9, atol=1e-12 * scale)
    np.testing.assert_allclose(dq, dq_o, rtol=1e-9, atol=1e-12 * np.abs(dq_o).max())
    g.close()


def test_adjoint_in_an_expanding_background():
    """With a scale factor the gradients are those of the proper-unit problem: the oracle's
    complex-step derivatives at proper cell size cell*a and density n_H*a^-3 (the
    derivative w.r.t. log n_HI is the same for comoving and proper densities)."""
    n = 12
    cell = 10 * S.KPC_CM
    a = 1.37
    nH, xHI, pos, ndot, R, w = _box(n, 43, 3e-3, 4)
    tab = O.make_table("bb")
    g = gpu_grid(n, cell, nH, xHI, pos, ndot, R, tab)
    g.set_scale_factor(a)
    dn, dq = g.backward(dev(w))
    dn, dq = dn.cpu().numpy(), dq.cpu().numpy()
    g.stats()
    cells = np.arange(n ** 3, dtype=np.int64)
    dn_o, dq_o = O.loss_grad_cs(n, cell * a, nH * (1.0 / (a * a * a)), xHI, pos, ndot, R, tab, w,
                                cells, np.arange(len(ndot)), nthreads=8)
    scale = np.abs(dn_o).max()
    assert scale > 0
    np.testing.assert_allclose(dn, dn_o, rtol=1e-9, atol=1e-12 * scale)
    np.testing.assert_allclose(dq, dq_o, rtol=1e-9, atol=1e-12 * np.abs(dq_o).max())
    g.close()


def _loss(g, w):
    gam = g.raytrace().cpu().numpy()
    return math.fsum(w * gam)


def test_adjoint_matches_central_differences_64cube():
    """64^3 box (0.78125 Mpc cells), 256 sources with R = 16, weights ~ N(0,1):
    central differences (step 1e-6 in log n_HI and log Ndot) of the GPU forward."""
    n = 64
    w_ = S.lognormal_box(n, 50.0, 256, 1e50, 1e54, radius=16.0)
    cell = w_["cell_cm"]
    nH = w_["nH"].reshape(-1)
    xHI = w_["xHI"].reshape(-1) * 1e-3  # partially ionised: rates reach many cells
    pos, ndot, R = w_["pos"], w_["ndot"], w_["radius"]
    w = S.loss_weights(n ** 3)
    tab = O.make_table("grey_exact")
    g = gpu_grid(n, cell, nH, xHI, pos, ndot, R, tab)
    dn, dq = g.backward(dev(w))
    dn = dn.cpu().numpy()
    dq = dq.cpu().numpy()
    rng = np.random.default_rng(3)
    near = [((int(p[0]) * n + int(p[1])) * n + int((p[2] + 2) % n)) for p in pos[:64]]
    cells = np.unique(np.concatenate([near, rng.integers(0, n ** 3, 64)]))
    h = 1e-6
    fd, ad = [], []
    nHd = dev(nH)
    for c in cells:
        v = nH[c]
        nHd[c] = v * math.exp(h)
        g.set_density(nHd)
        up = _loss(g, w)
        nHd[c] = v * math.exp(-h)
        g.set_density(nHd)
        dnn = _loss(g, w)
        nHd[c] = v
        fd.append((up - dnn) / (2 * h))
        ad.append(dn[c])
    g.set_density(nHd)
    fd, ad = np.array(fd), np.array(ad)
    assert np.linalg.norm(fd - ad) <= 1e-6 * np.linalg.norm(ad)
    fq = []
    for s in range(0, len(ndot), 8):
        q = ndot.copy()
        q[s] *= math.exp(h)
        g.set_sources(dev(pos, torch.int32), dev(q), dev(R))
        up = _loss(g, w)
        q[s] = ndot[s] * math.exp(-h)
        g.set_sources(dev(pos, torch.int32), dev(q), dev(R))
        fq.append((up - _loss(g, w)) / (2 * h))
    fq = np.array(fq)
    aq = dq[::8]
    assert np.linalg.norm(fq - aq) <= 1e-6 * np.linalg.norm(aq)
    g.close()


def test_autograd_function():
    from paper_2311_01492_gb300 import api
    n = 16
    cell = 10 * S.KPC_CM
    nH, xHI, pos, ndot, R, w = _box(n, 43, 1.0, 3)
    nhi = nH * xHI * 3e-3
    g = api.Grid(n, cell)
    g.set_tables("grey_exact")
    log_n = dev(np.log(nhi)).requires_grad_(True)
    log_q = dev(np.log(ndot)).requires_grad_(True)
    gam = api.raytrace_autograd(g, log_n, log_q, dev(pos, torch.int32), dev(R))
    loss = (gam * dev(w)).sum()
    loss.backward()
    tab = O.make_table("grey_exact")
    dn_o, dq_o = O.loss_grad_cs(n, cell, nhi, np.ones(n ** 3), pos, ndot, R, tab, w,
                                np.arange(n ** 3), np.arange(3), nthreads=8)
    np.testing.assert_allclose(log_n.grad.cpu().numpy(), dn_o, rtol=1e-9,
                               atol=1e-12 * np.abs(dn_o).max())
    np.testing.assert_allclose(log_q.grad.cpu().numpy(), dq_o, rtol=1e-9)
    g.close()
