"""Seeded generators for the synthetic wideband problems.

Shapes follow the paper's simulations (Sec. 4.1): an N = n x n image cube of
L channels spread linearly over a band, Gaussian-density uv sampling at the
reference frequency nu_0 scaled by nu_l / nu_0 for channel l, and additive
white complex Gaussian noise at a stated input SNR. The paper's W28 image and
VLA coverage are not available; Gaussian blobs with power-law spectra stand in
for the sources (rank <= number of blobs, as the mixture model implies).

Random streams: numpy Generator(PCG64(seed)), seed = 1000 * config + realisation.
Draw order inside one problem is fixed: blobs, spectra, diffuse field (if
any), uv holes (if any), uv pool, per-channel visibility counts (if uneven),
noise.
"""

from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np


# Workloads. "insnr" is the input SNR in dB, "uv_std" the per-axis standard
# deviation of the base coverage in radians at nu_0, "uv_limit" the band edge
# (max |u|, |v| after scaling to the highest channel), "M" either a count per
# channel or a (lo, hi) range drawn uniformly per channel.
CONFIGS = {
    1: dict(name="C1 64x64 L=4 M=2000 fp64", n=64, L=4, f_lo=1.0, f_hi=2.0, M=2000,
            Q=3, insnr=40.0, uv_std=np.pi / 4, uv_limit=np.pi, iters=200, prec="f64"),
    2: dict(name="C2 256x256 L=60 M=32768 fp32", n=256, L=60, f_lo=1.0, f_hi=2.0, M=32768,
            Q=3, insnr=40.0, uv_std=np.pi / 4, uv_limit=np.pi, iters=500, prec="f32"),
    3: dict(name="C3 512x512 L=32 M~U[1e5,4e5] fp32", n=512, L=32, f_lo=1.0, f_hi=2.0,
            M=(100_000, 400_000), Q=3, insnr=40.0, uv_std=np.pi / 4, uv_limit=np.pi,
            iters=50, prec="f32"),
    4: dict(name="C4 1024x1024 L=16 M=1e6 fp32", n=1024, L=16, f_lo=1.0, f_hi=2.0,
            M=1_000_000, Q=50, insnr=30.0, uv_std=np.pi / 4, uv_limit=0.9 * np.pi,
            diffuse=True, iters=100, prec="f32"),
    5: dict(name="C5 2048x2048 L=64 M~U[5e5,2e6] fp32", n=2048, L=64, f_lo=1.0, f_hi=4.0,
            M=(500_000, 2_000_000), Q=3, insnr=40.0, uv_std=np.pi / 4, uv_limit=np.pi,
            iters=100, prec="f32"),
}


@dataclass
class ProblemInputs:
    """Random inputs of one synthetic wideband problem (no derived quantities)."""

    nx: int
    ny: int
    freqs: np.ndarray            # (L,) channel frequencies (GHz), freqs[0] = nu_0
    truth: np.ndarray            # (L, ny, nx) float64, max = 1, >= 0
    uv: np.ndarray               # (sum M, 2) float64 radians, channel-concatenated
    offsets: np.ndarray          # (L + 1,) int64 visibility offsets per channel
    noise: np.ndarray            # (sum M,) complex128, unit variance complex normal
    insnr: float                 # input SNR in dB
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def L(self) -> int:
        return int(self.truth.shape[0])

    @property
    def M(self) -> np.ndarray:
        return np.diff(self.offsets)


def channel_freqs(L: int, f_lo: float, f_hi: float) -> np.ndarray:
    """Channels spaced linearly over [f_lo, f_hi]; a single channel sits at f_lo."""
    if L == 1:
        return np.array([f_lo], dtype=np.float64)
    return np.linspace(f_lo, f_hi, L)


def gaussian_blobs(rng, nx: int, ny: int, Q: int, sigma_range=(2.0, 5.0),
                   amp_range=(0.5, 1.0)) -> np.ndarray:
    """Q isotropic Gaussian sources, centres uniform inside a 3-sigma margin.

    Returns S as (Q, ny, nx). On images smaller than 41 pixels the width range
    is narrowed so that the margin still fits."""
    s_hi = min(sigma_range[1], (min(nx, ny) - 1) / 8.0)
    s_lo = min(sigma_range[0], s_hi)
    sig = rng.uniform(s_lo, s_hi, Q)
    cx = rng.uniform(3 * sig, nx - 1 - 3 * sig)
    cy = rng.uniform(3 * sig, ny - 1 - 3 * sig)
    amp = rng.uniform(amp_range[0], amp_range[1], Q)
    yy, xx = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                         indexing="ij")
    S = np.empty((Q, ny, nx))
    for q in range(Q):
        S[q] = amp[q] * np.exp(-((xx - cx[q]) ** 2 + (yy - cy[q]) ** 2) / (2.0 * sig[q] ** 2))
    return S


def power_law_spectra(rng, freqs: np.ndarray, Q: int, index_range=(-1.0, 1.0)) -> np.ndarray:
    """Spectra h_q(nu) = (nu / nu_0)^(-alpha_q), alpha_q uniform. Returns H (L, Q)."""
    alpha = rng.uniform(index_range[0], index_range[1], Q)
    ratio = freqs / freqs[0]
    return ratio[:, None] ** (-alpha[None, :])


def diffuse_field(rng, nx: int, ny: int, slope: float = 1.5, peak: float = 0.1) -> np.ndarray:
    """Positive Gaussian-random-field image: white noise filtered by |k|^-slope,
    exponentiated and scaled to the given peak."""
    white = rng.standard_normal((ny, nx))
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.fftfreq(nx)[None, :]
    kk = np.sqrt(kx ** 2 + ky ** 2)
    kk[0, 0] = np.inf
    field_ = np.fft.ifft2(np.fft.fft2(white) * kk ** (-slope)).real
    field_ = (field_ - field_.mean()) / (field_.std() + 1e-300)
    img = np.exp(field_)
    return peak * img / img.max()


def uv_holes(rng, n_holes: int, std: float, limit: float, scale_max: float):
    """Holes of the sampling function (Sec. 4.1: an inverse Gaussian profile, so
    that the missing Fourier content sits mainly at high spatial frequencies).
    Reading: n_holes discs at nu_0 whose centres are drawn inside the band with
    density proportional to 1 - exp(-|c|^2 / (2 std^2)) (rejection sampling),
    radii uniform in [0.04, 0.12] * limit / scale_max.

    Returns (centres (n_holes, 2), radii (n_holes,))."""
    edge = limit / scale_max
    cs = np.empty((0, 2))
    while cs.shape[0] < n_holes:
        c = rng.uniform(-edge, edge, size=(4 * n_holes + 16, 2))
        accept = rng.uniform(0.0, 1.0, size=c.shape[0]) < 1.0 - np.exp(-np.sum(c * c, axis=1) / (2 * std * std))
        cs = np.concatenate([cs, c[accept]], axis=0)
    cs = cs[:n_holes]
    radii = rng.uniform(0.04, 0.12, size=n_holes) * edge
    return cs, radii


def in_holes(pts: np.ndarray, centres: np.ndarray, radii: np.ndarray) -> np.ndarray:
    """True for the points (K, 2) inside any hole."""
    if centres.shape[0] == 0:
        return np.zeros(pts.shape[0], dtype=bool)
    d2 = np.sum((pts[:, None, :] - centres[None, :, :]) ** 2, axis=2)
    return np.any(d2 < radii[None, :] ** 2, axis=1)


def uv_coverage(rng, M_max: int, freqs: np.ndarray, std: float, limit: float,
                holes: int = 0) -> np.ndarray:
    """Base coverage at nu_0: i.i.d. N(0, std^2) per axis, rejecting points that
    would leave the band [-limit, limit) once scaled to the highest channel and,
    with holes > 0, points inside the holes of uv_holes (drawn first).

    Returns the (M_max, 2) base pool at nu_0; channel l uses pool[:M_l] * nu_l / nu_0."""
    scale_max = freqs[-1] / freqs[0]
    centres, radii = (uv_holes(rng, holes, std, limit, scale_max) if holes > 0
                      else (np.zeros((0, 2)), np.zeros(0)))
    out = np.empty((0, 2))
    while out.shape[0] < M_max:
        need = M_max - out.shape[0]
        draw = rng.normal(0.0, std, size=(int(need * 1.3) + 16, 2))
        keep = (np.max(np.abs(draw), axis=1) * scale_max < limit) & ~in_holes(draw, centres, radii)
        out = np.concatenate([out, draw[keep]], axis=0)
    return out[:M_max]


def noise_draws(rng, n: int) -> np.ndarray:
    """Unit-variance complex normal draws (N(0,1) + i N(0,1)) / sqrt(2)."""
    re = rng.standard_normal(n)
    im = rng.standard_normal(n)
    return (re + 1j * im) / np.sqrt(2.0)


def make_inputs(config: int | dict, realisation: int = 0, *, n: int | None = None,
                L: int | None = None, M=None, Q: int | None = None, seed: int | None = None,
                insnr: float | None = None, f_lo: float | None = None,
                f_hi: float | None = None, holes: int | None = None) -> ProblemInputs:
    """Draw one problem. Keyword arguments override the configuration's sizes
    (used for reduced parity cases of a configuration's generator)."""
    if isinstance(config, int):
        cfg = dict(CONFIGS[config])
        cfg_id = config
    else:
        cfg = dict(config)
        cfg_id = int(cfg.get("id", 0))
    if n is not None:
        cfg["n"] = n
    if L is not None:
        cfg["L"] = L
    if M is not None:
        cfg["M"] = M
    if Q is not None:
        cfg["Q"] = Q
    if insnr is not None:
        cfg["insnr"] = insnr
    if f_lo is not None:
        cfg["f_lo"] = f_lo
    if f_hi is not None:
        cfg["f_hi"] = f_hi
    if holes is not None:
        cfg["holes"] = holes
    if seed is None:
        seed = 1000 * cfg_id + realisation
    rng = np.random.Generator(np.random.PCG64(seed))
    nx = ny = int(cfg["n"])
    Lc = int(cfg["L"])
    freqs = channel_freqs(Lc, cfg["f_lo"], cfg["f_hi"])

    S = gaussian_blobs(rng, nx, ny, int(cfg["Q"]))
    H = power_law_spectra(rng, freqs, int(cfg["Q"]))
    # X = S H^T: pixels x channels, stored channel-major (L, ny, nx).
    X = np.einsum("qyx,lq->lyx", S, H)
    if cfg.get("diffuse"):
        D = diffuse_field(rng, nx, ny)
        hd = power_law_spectra(rng, freqs, 1)[:, 0]
        X = X + hd[:, None, None] * D[None]
    X = X / X.max()

    Mspec = cfg["M"]
    if isinstance(Mspec, (tuple, list)):
        M_max = int(Mspec[1])
    else:
        M_max = int(Mspec)
    pool = uv_coverage(rng, M_max, freqs, float(cfg["uv_std"]), float(cfg["uv_limit"]),
                       holes=int(cfg.get("holes", 0)))
    if isinstance(Mspec, (tuple, list)):
        Ml = rng.integers(int(Mspec[0]), int(Mspec[1]) + 1, size=Lc)
    else:
        Ml = np.full(Lc, int(Mspec))
    offsets = np.zeros(Lc + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(Ml)
    uv = np.empty((int(offsets[-1]), 2))
    for l in range(Lc):
        uv[offsets[l]:offsets[l + 1]] = pool[:Ml[l]] * (freqs[l] / freqs[0])
    noise = noise_draws(rng, int(offsets[-1]))
    return ProblemInputs(nx=nx, ny=ny, freqs=freqs, truth=X, uv=uv, offsets=offsets,
                         noise=noise, insnr=float(cfg["insnr"]), seed=int(seed),
                         meta=dict(config=cfg_id, name=cfg.get("name", ""), iters=cfg.get("iters"),
                                   prec=cfg.get("prec")))
