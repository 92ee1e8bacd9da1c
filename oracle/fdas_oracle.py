"""FP64 CPU oracle of the Fourier Domain Acceleration Search hot path.

TEST INFRASTRUCTURE, NOT PRODUCT CODE. Only the test suite, the smoke check
in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import
this module. It shares no code with the CUDA path and is deliberately plain
and slow: whole-array numpy/scipy steps in float64, in the order the paper
gives them (Section 4, steps 2-7), followed by the harmonic sum and the
threshold that the search adds after the power plane.

Pins: every function here is checked in ``tests/test_oracle_pins.py``
against something other than itself (closed forms, brute force on tiny
inputs, Euler-Maclaurin error terms, invariants); see the docstrings.

Readings of the paper used here (the paper is silent or garbled on them):
  * Eq. 1 has m+1 terms and a garbled index; the plane is read as m taps,
    A(r, z) = sum_{d=-m/2}^{m/2-1} Xw[r+d] * tau_z(d).
  * tau_z is the conjugated response of a constant-acceleration signal whose
    *mean* frequency is r (template centred on d = 0), Section 2; z = fdot T^2
    with T the observation length.
  * the spectrum keeps bins 0..N/2-1 (Nyquist dropped); whitening is a
    64-bin running median (the step is not in the paper). The block-median
    variant takes medians of consecutive 64-bin blocks from bin 1, places
    them at the block centres and interpolates linearly between centres
    (constant beyond the first and last centre).
  * harmonic sums use round-half-up in r and round-half-away-from-zero in
    the centred z index; the threshold is the Gamma(h, 1) tail that equals
    the one-sided Gaussian tail at ``sigma``.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import optimize, special

LN2 = math.log(2.0)
MEDIAN_WINDOW = 64


# ----------------------------------------------------------------------------
# Grid helpers (Section 2: z = fdot * T^2 templates, spaced dz apart)
# ----------------------------------------------------------------------------
def n_templates(zmax: int, dz: int) -> int:
    return 2 * (zmax // dz) + 1


def z_values(zmax: int, dz: int) -> np.ndarray:
    return -zmax + dz * np.arange(n_templates(zmax, dz), dtype=np.float64)


# ----------------------------------------------------------------------------
# Step 2 (Section 4): real-to-complex DFT of the series.
# ----------------------------------------------------------------------------
def spectrum(x: np.ndarray) -> np.ndarray:
    """X_k = sum_n x_n exp(-2 pi i k n / N), k = 0 .. N/2-1 (Nyquist dropped).

    numpy's FFT is the library step; pinned against a direct DFT sum.
    """
    x = np.asarray(x, dtype=np.float64)
    return np.fft.rfft(x)[: x.shape[0] // 2]


# ----------------------------------------------------------------------------
# Spectral whitening (not in the paper; added by the search contract).
# ----------------------------------------------------------------------------
def window_start(k: np.ndarray, nb: int, w: int = MEDIAN_WINDOW) -> np.ndarray:
    """First bin of the w-bin median window of bin k: [k-w/2, k+w/2-1],
    shifted (not shrunk) so that it lies inside [1, nb-1]."""
    return np.clip(np.asarray(k) - w // 2, 1, nb - w)


def running_median_power(X: np.ndarray, w: int = MEDIAN_WINDOW) -> np.ndarray:
    """mu_k = even-count median (mean of the two middle order statistics) of
    |X|^2 over the window of bin k; mu_0 is unused (returned as nan)."""
    nb = X.shape[0]
    if nb < w + 1:
        raise ValueError("spectrum too short for the median window")
    p = np.abs(X) ** 2
    n_starts = nb - w                     # starts 1 .. nb-w
    med = np.empty(n_starts + 1)
    med[0] = np.nan
    view = np.lib.stride_tricks.sliding_window_view(p[1:], w)  # rows = starts
    chunk = 1 << 16
    for a in range(0, n_starts, chunk):
        b = min(a + chunk, n_starts)
        part = np.partition(view[a:b], [w // 2 - 1, w // 2], axis=1)
        med[1 + a: 1 + b] = 0.5 * (part[:, w // 2 - 1] + part[:, w // 2])
    mu = np.empty(nb)
    mu[0] = np.nan
    k = np.arange(1, nb)
    mu[1:] = med[window_start(k, nb, w)]
    return mu


def whiten(X: np.ndarray, w: int = MEDIAN_WINDOW) -> np.ndarray:
    """Xw_k = X_k * sqrt(ln 2 / mu_k), Xw_0 = 0.

    For complex Gaussian noise |X|^2 is exponential and its median is
    ln 2 times its mean, so whitened noise has unit mean power.
    """
    mu = running_median_power(X, w)
    Xw = np.zeros_like(X, dtype=np.complex128)
    Xw[1:] = X[1:] * np.sqrt(LN2 / mu[1:])
    return Xw


def block_median_power(X: np.ndarray, w: int = MEDIAN_WINDOW) -> np.ndarray:
    """mu_k of the block-median variant: the textbook median of |X|^2 over
    each block [1 + w b, min(1 + w (b+1), nb)) (the last block may be short),
    placed at the block centre c_b = (first + last) / 2, then linear
    interpolation in k between adjacent centres and the end medians beyond
    the first and last centre; mu_0 is unused (nan)."""
    nb = X.shape[0]
    if nb < w + 1:
        raise ValueError("spectrum too short for the median block")
    p = np.abs(X) ** 2
    starts = np.arange(1, nb, w)
    ends = np.minimum(starts + w, nb)
    med = np.array([np.median(p[a:b]) for a, b in zip(starts, ends)])
    cen = 0.5 * (starts + ends - 1)
    mu = np.interp(np.arange(nb, dtype=np.float64), cen, med)
    mu[0] = np.nan
    return mu


def whiten_block(X: np.ndarray, w: int = MEDIAN_WINDOW) -> np.ndarray:
    """Xw_k = X_k * sqrt(ln 2 / mu_k) with the block-median mu; Xw_0 = 0."""
    mu = block_median_power(X, w)
    Xw = np.zeros_like(X, dtype=np.complex128)
    Xw[1:] = X[1:] * np.sqrt(LN2 / mu[1:])
    return Xw


# ----------------------------------------------------------------------------
# Templates (Section 2; the response of Ransom et al. 2002, which Eq. 1 uses)
# ----------------------------------------------------------------------------
def template_fresnel(z: float, m: int, offset: float = 0.0) -> np.ndarray:
    """tau_z(d) = int_0^1 exp(2 pi i [(d - offset + z/2) u - z u^2 / 2]) du for
    d = -m/2 .. m/2-1, via the Fresnel integrals C, S (scipy, float64).
    ``offset`` evaluates the response at a fractional frequency r + offset.

    Completing the square with q = d - offset + z/2, s_a = sqrt(2|z|)(a - q/z):
        tau = conj( exp(-i pi q^2/z) [dC + i sgn(z) dS] ) / sqrt(2|z|),
    dC = C(s_1) - C(s_0), dS = S(s_1) - S(s_0). For z = 0 the integral is
    (exp(2 pi i q) - 1) / (2 pi i q), i.e. delta_{d,0} at zero offset.
    """
    d = np.arange(-m // 2, m // 2, dtype=np.float64)
    if z == 0:
        q = d - offset
        out = np.ones(m, dtype=np.complex128)
        nz = q != 0
        out[nz] = (np.exp(2j * np.pi * q[nz]) - 1.0) / (2j * np.pi * q[nz])
        if offset == 0.0:
            out = (d == 0).astype(np.complex128)
        return out
    q = d - offset + z / 2.0
    scale = math.sqrt(2.0 * abs(z))
    s0 = scale * (0.0 - q / z)
    s1 = scale * (1.0 - q / z)
    S0, C0 = special.fresnel(s0)
    S1, C1 = special.fresnel(s1)
    dF = (C1 - C0) + 1j * np.sign(z) * (S1 - S0)
    # exp(-i pi q^2 / z) with the argument reduced exactly: q^2/z = Q^2/(4z),
    # Q = 2q an integer whenever z is an integer.
    Q = np.rint(2.0 * q).astype(np.int64)
    if offset == 0.0 and float(z).is_integer():
        zi = int(z)
        red = np.mod(Q * Q, 8 * abs(zi)) / (4.0 * abs(zi))     # in [0, 2)
        ph = np.exp(-1j * np.pi * red * np.sign(zi))
    else:
        ph = np.exp(-1j * np.pi * q * q / z)
    return np.conj(ph * dF) / scale


def template_discrete(z: float, m: int, n: int) -> np.ndarray:
    """Exact DFT-domain response of a sampled chirp of length n:
    tau_z(d) = (1/n) sum_k exp(2 pi i [(d + z/2) k/n - z k^2/(2 n^2)]),
    for d = -m/2 .. m/2-1 (one float64 inverse FFT of the chirp)."""
    k = np.arange(n, dtype=np.float64)
    cyc = (z / 2.0) * k / n - z * k * k / (2.0 * n * n)
    cyc -= np.floor(cyc)
    u = np.exp(2j * np.pi * cyc)
    t = np.fft.ifft(u)
    d = np.arange(-m // 2, m // 2)
    return t[np.mod(d, n)]


def template_bank(zmax: int, dz: int, m: int, offset: float = 0.0) -> np.ndarray:
    """(Z, m) complex128 taps tau_{z_j}(d), rows j = 0..Z-1, z_j = -zmax + j dz
    (at the fractional frequency offset ``offset``)."""
    return np.stack([template_fresnel(z, m, offset) for z in z_values(zmax, dz)])


# ----------------------------------------------------------------------------
# Steps 3-7 (Section 4) as their definition: the f-fdot power plane.
# ----------------------------------------------------------------------------
def correlate_row(Xw: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """A(r) = sum_{d=-m/2}^{m/2-1} Xw[r+d] tau(d), r = 0..nb-1, Xw = 0 outside
    [0, nb). One zero-padded FFT correlation over the whole spectrum (no
    segmenting): FFT(A) = FFT(Xw_pad) * conj(FFT(conj(g))), g[d mod Lc] = tau(d).
    """
    nb = Xw.shape[0]
    m = tau.shape[0]
    lc = 1
    while lc < nb + m:
        lc *= 2
    a = np.zeros(lc, dtype=np.complex128)
    a[:nb] = Xw
    g = np.zeros(lc, dtype=np.complex128)
    d = np.arange(-m // 2, m // 2)
    g[np.mod(d, lc)] = tau
    c = np.fft.ifft(np.fft.fft(a) * np.conj(np.fft.fft(np.conj(g)))) * 1.0
    return c[:nb]


def power_plane(Xw: np.ndarray, taus: np.ndarray) -> np.ndarray:
    """P[j, r] = |A_j(r)|^2, shape (Z, nb), float64 (step 7: powers)."""
    return np.stack([np.abs(correlate_row(Xw, t)) ** 2 for t in taus])


def power_plane_interbin(Xw: np.ndarray, zmax: int, dz: int, m: int) -> np.ndarray:
    """The half-bin plane: P2[j, 2r + e] = |A(r + e/2, z_j)|^2, e = 0, 1, with
    A(r + 1/2, z) = sum_d Xw[r+d] tau_z(d) at offset 1/2 (the same m taps
    d = -m/2 .. m/2-1 around bin r); shape (Z, 2 nb), columns in half bins."""
    P0 = power_plane(Xw, template_bank(zmax, dz, m))
    P1 = power_plane(Xw, template_bank(zmax, dz, m, offset=0.5))
    P2 = np.empty((P0.shape[0], 2 * P0.shape[1]))
    P2[:, 0::2] = P0
    P2[:, 1::2] = P1
    return P2


def plane_cells(Xw: np.ndarray, taus: np.ndarray, j_idx, r_idx) -> np.ndarray:
    """Direct sums of Eq. 1 at individual cells (j, r): for full-size checks."""
    nb = Xw.shape[0]
    m = taus.shape[1]
    d = np.arange(-m // 2, m // 2)
    j_idx = np.asarray(j_idx)
    r_idx = np.asarray(r_idx)
    out = np.empty(j_idx.shape[0])
    for i, (j, r) in enumerate(zip(j_idx, r_idx)):
        idx = r + d
        ok = (idx >= 0) & (idx < nb)
        out[i] = abs(np.sum(Xw[idx[ok]] * taus[j][ok])) ** 2
    return out


# ----------------------------------------------------------------------------
# Harmonic sum and threshold (added after step 7 by the search contract).
# ----------------------------------------------------------------------------
def harmonic_levels(nharm: int):
    out, h = [], 1
    while h <= nharm:
        out.append(h)
        h *= 2
    return out


def subharmonic_r(r, k: int, h: int):
    """round(k r / h), ties up: floor((2 k r + h) / (2 h))."""
    return (2 * k * np.asarray(r, dtype=np.int64) + h) // (2 * h)


def subharmonic_j(j, k: int, h: int, zc: int):
    """zc + round(k (j - zc) / h), ties away from zero (keeps z symmetry)."""
    jc = np.asarray(j, dtype=np.int64) - zc
    a = np.abs(k * jc)
    return zc + np.sign(jc) * ((2 * a + h) // (2 * h))


def harmonic_sums(P: np.ndarray, nharm: int) -> dict:
    """H_h[j, r] = sum_{k=1..h} P[jz(k, j, h), rr(k, r, h)] for h = 1, 2, 4..nharm."""
    Z, nb = P.shape
    zc = (Z - 1) // 2
    r = np.arange(nb)
    j = np.arange(Z)
    out = {}
    for h in harmonic_levels(nharm):
        H = np.zeros_like(P)
        for k in range(1, h + 1):
            H += P[np.ix_(subharmonic_j(j, k, h, zc), subharmonic_r(r, k, h))]
        out[h] = H
    return out


def gaussian_tail(sigma: float) -> float:
    """One-sided Gaussian tail probability of a sigma-sigma excess."""
    return 0.5 * math.erfc(sigma / math.sqrt(2.0))


def thresholds(nharm: int, sigma: float = 6.0) -> dict:
    """T_h with P(Gamma(h, 1) >= T_h) = gaussian_tail(sigma): the sum of h
    whitened noise powers (each exponential with unit mean) is Gamma(h, 1)."""
    p = gaussian_tail(sigma)
    return {h: float(special.gammainccinv(h, p)) for h in harmonic_levels(nharm)}


def candidates(P: np.ndarray, nharm: int, sigma: float = 6.0):
    """All (r, j, h, H) with r >= 1 and H_h(r, j) >= T_h, sorted by (h, r, j)."""
    T = thresholds(nharm, sigma)
    H = harmonic_sums(P, nharm)
    rows = []
    for h in harmonic_levels(nharm):
        jj, rr = np.nonzero(H[h][:, 1:] >= T[h])
        rr = rr + 1
        for a, b in zip(rr, jj):
            rows.append((int(a), int(b), h, float(H[h][b, a])))
    rows.sort(key=lambda t: (t[2], t[0], t[1]))
    return rows, H


# ----------------------------------------------------------------------------
# Candidate distillation (after the threshold; not in the paper).
# ----------------------------------------------------------------------------
def log_gamma_tail(h: int, x: float) -> float:
    """ln Q(h, x), the Gamma(h, 1) upper tail for integer h in its Poisson
    form Q = exp(-x) sum_{k<h} x^k / k!, which does not underflow."""
    s, term = 0.0, 1.0
    for k in range(h):
        if k > 0:
            term *= x / k
        s += term
    return -x + math.log(s)


def gaussian_sigma(log_p: float) -> float:
    """The s with ln Phi_bar(s) = log_p (one-sided Gaussian tail): a bracketed
    root of scipy's log_ndtr(-s) - log_p."""
    def f(s):
        return float(special.log_ndtr(-s)) - log_p
    hi = 40.0
    while f(hi) > 0:
        hi *= 2.0
    return float(optimize.brentq(f, -40.0, hi, xtol=1e-13, rtol=1e-15))


def distill(rows, Z: int):
    """Local maxima of a candidate list ``rows`` of (r, j, h, H):
      * within level h, no candidate at (r + dr, j + dj), |dr|, |dj| <= 1,
        has a larger H (equal H: the smaller (j, r) wins);
      * across adjacent levels, candidates (r, jc) at level h and (r', jc') at
        level 2h are the same signal when |r' - 2r| <= 2 and |jc' - 2 jc| <= 2
        (jc = j - zc, zc = (Z-1)/2; a symmetric relation), and the one with
        the larger sigma wins (equal sigma: the lower level).
    Returns (r, j, h, H, sigma, log10 p) rows sorted by (h, r, j), with sigma
    the Gaussian-equivalent significance of H under Gamma(h, 1) noise and
    p = Q(h, H)."""
    zc = (Z - 1) // 2
    H = {(r, j, h): float(v) for (r, j, h, v) in rows}
    lp = {key: log_gamma_tail(key[2], v) for key, v in H.items()}
    sg = {key: gaussian_sigma(v) for key, v in lp.items()}
    out = []
    for (r, j, h), v in H.items():
        me = (r, j, h)
        keep = True
        for (r2, j2, h2), w in H.items():
            if h2 == h:
                if max(abs(r2 - r), abs(j2 - j)) == 1 and (w > v or (w == v and (j2, r2) < (j, r))):
                    keep = False
            elif h2 == 2 * h or 2 * h2 == h:
                lo, hi = ((r, j - zc), (r2, j2 - zc)) if h2 > h else ((r2, j2 - zc), (r, j - zc))
                if abs(hi[0] - 2 * lo[0]) <= 2 and abs(hi[1] - 2 * lo[1]) <= 2:
                    if sg[(r2, j2, h2)] > sg[me] or (sg[(r2, j2, h2)] == sg[me] and h2 < h):
                        keep = False
        if keep:
            out.append((r, j, h, v, sg[me], lp[me] / math.log(10.0)))
    out.sort(key=lambda t: (t[2], t[0], t[1]))
    return out


def correlate_band(Xw: np.ndarray, tau: np.ndarray, c0: int, c1: int) -> np.ndarray:
    """A(r) = sum_{d=-m/2}^{m/2-1} Xw[r+d] tau(d) for r = c0 .. c1-1 only, Xw = 0
    outside [0, nb): one zero-padded FFT correlation of the sub-band
    Xw[c0 - m/2, c1 + m/2) (the same definition as correlate_row, restricted
    to a column range, so that full-size checks need not form whole rows)."""
    nb = Xw.shape[0]
    m = tau.shape[0]
    lo = c0 - m // 2
    width = (c1 - c0) + m
    band = np.zeros(width, dtype=np.complex128)
    a, b = max(lo, 0), min(lo + width, nb)
    if b > a:
        band[a - lo: b - lo] = Xw[a:b]
    # band[i] = Xw[lo + i]; A(c0 + t) = sum_d band[t + m/2 + d] tau(d)
    full = correlate_row(band, tau)
    return full[m // 2: m // 2 + (c1 - c0)]


def subharmonic_fractions(nharm: int):
    """The distinct ratios k/h (k = 1..h, h = 1, 2, 4..nharm) as (q, Q) with
    k/h = q/Q, Q = nharm: round(k r / h) depends on k/h alone."""
    return [(q, nharm) for q in range(1, nharm + 1)]


def harmonic_sums_window(Xw: np.ndarray, taus: np.ndarray, nharm: int, r_a: int, r_b: int) -> dict:
    """H_h[j, r - r_a] for every row j and the top bins r_a <= r < r_b, with
    the plane formed only where these sums read it: for each ratio k/h the
    columns round(k r / h), r in [r_a, r_b), of every row, by correlate_band.
    Same definition and summation order (k = 1..h) as harmonic_sums."""
    Z = taus.shape[0]
    zc = (Z - 1) // 2
    r = np.arange(r_a, r_b, dtype=np.int64)
    j = np.arange(Z)
    bands = {}
    for q, Q in subharmonic_fractions(nharm):
        cols = subharmonic_r(r, q, Q)
        c0, c1 = int(cols.min()), int(cols.max()) + 1
        rows = np.stack([np.abs(correlate_band(Xw, t, c0, c1)) ** 2 for t in taus])
        bands[(q, Q)] = (c0, rows)
    out = {}
    for h in harmonic_levels(nharm):
        H = np.zeros((Z, r_b - r_a))
        for k in range(1, h + 1):
            q, Q = k * nharm // h, nharm
            c0, rows = bands[(q, Q)]
            H += rows[np.ix_(subharmonic_j(j, k, h, zc), subharmonic_r(r, k, h) - c0)]
        out[h] = H
    return out


def harmonic_sum_cells(Xw, taus, nharm: int, j_idx, r_idx) -> dict:
    """H_h at individual top cells from direct plane-cell sums (full-size checks)."""
    Z = taus.shape[0]
    zc = (Z - 1) // 2
    out = {}
    for h in harmonic_levels(nharm):
        acc = np.zeros(len(j_idx))
        for k in range(1, h + 1):
            acc += plane_cells(Xw, taus, subharmonic_j(j_idx, k, h, zc),
                               subharmonic_r(r_idx, k, h))
        out[h] = acc
    return out


# ----------------------------------------------------------------------------
# The whole path on one series.
# ----------------------------------------------------------------------------
def search(x: np.ndarray, zmax: int, dz: int, m: int, nharm: int,
           sigma: float = 6.0, whitening: str = "running", interbin: bool = False):
    """Returns (Xw, taus, P, candidate rows, harmonic sums); ``whitening`` is
    "running" (64-bin running median) or "block" (block-median variant);
    with ``interbin`` the plane is the half-bin plane and every r (plane
    column, candidate r_top) counts half bins."""
    X = spectrum(x)
    Xw = whiten(X) if whitening == "running" else whiten_block(X)
    taus = template_bank(zmax, dz, m)
    P = power_plane_interbin(Xw, zmax, dz, m) if interbin else power_plane(Xw, taus)
    cands, H = candidates(P, nharm, sigma)
    return Xw, taus, P, cands, H
