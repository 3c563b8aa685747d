"""Binned power spectrum and cross-correlation coefficient (oracle, float64).

Sec. 3.1 uses the baryon power spectrum (estimator deferred to another paper); Sec. 3.2
uses r_c(k) = P_XY / sqrt(P_XX P_YY). Reading used here: bins of width k_f = 2 pi / L with
bin index round(|k| / k_f) (bin 0 holds only k = 0 and is not reported), the half-complex
spectrum counted twice for 0 < k_x < N/2, and P = L^3 <|delta_k|^2> / N^6 with numpy FFT
normalisation. Bins 1..nbins are returned (mode-weighted mean |k|, P, number of modes).
"""
from __future__ import annotations

import numpy as np
import torch

from .pm import wavenumbers

_DT = torch.float64


def power_spectrum(a, box: float, nbins: int | None = None, b=None):
    n = a.shape[-1]
    nbins = nbins or n
    ak = torch.fft.rfftn(a, dim=(-3, -2, -1))
    bk = ak if b is None else torch.fft.rfftn(b, dim=(-3, -2, -1))
    power = (ak * bk.conj()).real
    (kx, ky, kz), _ = wavenumbers(n, box)
    kmag = torch.sqrt(kx ** 2 + ky ** 2 + kz ** 2).expand_as(power)
    kf = 2.0 * np.pi / box
    idx = torch.round(kmag / kf).to(torch.int64)
    w = torch.full((n // 2 + 1,), 2.0, dtype=_DT)
    w[0] = 1.0
    if n % 2 == 0:
        w[-1] = 1.0
    w = w.reshape(1, 1, -1).expand_as(power)
    keep = (idx >= 1) & (idx <= nbins)
    bi = idx[keep] - 1
    nm = torch.zeros(nbins, dtype=_DT).index_add(0, bi, w[keep])
    ks = torch.zeros(nbins, dtype=_DT).index_add(0, bi, (w * kmag)[keep])
    ps = torch.zeros(nbins, dtype=_DT).index_add(0, bi, (w * power)[keep])
    nz = nm > 0
    safe = torch.where(nz, nm, torch.ones_like(nm))
    kmean = torch.where(nz, ks / safe, torch.zeros_like(ks))
    pk = torch.where(nz, ps / safe, torch.zeros_like(ps)) * box ** 3 / n ** 6
    return kmean, pk, nm


def cross_correlation(x, y, box: float, nbins: int | None = None):
    _, pxy, nm = power_spectrum(x, box, nbins, y)
    _, pxx, _ = power_spectrum(x, box, nbins)
    _, pyy, _ = power_spectrum(y, box, nbins)
    ok = (pxx > 0) & (pyy > 0)
    return torch.where(ok, pxy / torch.sqrt(torch.where(ok, pxx * pyy, torch.ones_like(pxx))),
                       torch.zeros_like(pxy))
