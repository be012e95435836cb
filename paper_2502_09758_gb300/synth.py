"""Seeded synthetic inputs shaped like the paper's deblurring workloads.

This module only draws data: piecewise-constant test images, blur kernels and
noisy blurred observations.  It holds none of the solver's arithmetic and is
shared by the tests, the benchmark and the oracle checks as the one common
source of inputs.  The paper's own photographs (300 x 400 x 3, Sec. 4.2) and
1D signal (Sec. 4.1) are not available; these generators stand in for them.

Recipe (all draws from ``numpy.random.default_rng(seed)``):

* image: background 0.5*U per channel; ``12*sqrt(HW/64^2)`` axis-aligned
  rectangles and ``8*sqrt(HW/64^2)`` disks, uniform positions, sizes in
  ``[sqrt(HW)/16, sqrt(HW)/3]``, values U[0,1] (independent per channel),
  painted in order; optionally a smooth ramp ``0.2*(i/H + j/W)/2`` and texture
  noise U[-0.05, 0.05]; clipped to [0, 1].
* kernels: normalised Gaussians; motion blur as a centred segment of length L
  at angle theta, rasterised with 64-point supersampling and bilinear
  splatting, normalised; optional positive perturbation.
* observation: ``y = b_true (*) x + N(0, sigma^2)`` with periodic boundary,
  formed in float64 through NumPy's FFT (data synthesis only).
* 1D signal (Sec. 4.1's setting): length n, zero background with
  ``max(3, n // 32)`` boxes (uniform start, length U{n/32 .. n/8}, height
  U[0.2, 1]) and ``max(2, n // 64)`` single spikes (height U[0.3, 1]), painted
  in order; the forward matrix A is the Gaussian convolution with sigma = 5,
  the kernel cut at +-3 sigma and normalised to sum 1, zero outside the
  signal; ``y = A x + N(0, 0.005^2)``; the learned operator starts at B_0 = A.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def piecewise_image(rng, C, H, W, texture=False):
    HW = H * W
    scale = np.sqrt(HW / 64.0 ** 2)
    n_rect, n_disk = int(round(12 * scale)), int(round(8 * scale))
    smin, smax = np.sqrt(HW) / 16.0, np.sqrt(HW) / 3.0
    img = np.empty((C, H, W))
    img[:] = (0.5 * rng.uniform(size=C))[:, None, None]
    ii, jj = np.mgrid[0:H, 0:W]
    shapes = []
    for _ in range(n_rect):
        shapes.append(("rect", rng.uniform(0, H), rng.uniform(0, W),
                       rng.uniform(smin, smax), rng.uniform(smin, smax), rng.uniform(size=C)))
    for _ in range(n_disk):
        shapes.append(("disk", rng.uniform(0, H), rng.uniform(0, W),
                       rng.uniform(smin, smax) / 2.0, 0.0, rng.uniform(size=C)))
    for kind, ci, cj, s1, s2, val in shapes:
        if kind == "rect":
            m = (np.abs(ii - ci) <= s1 / 2) & (np.abs(jj - cj) <= s2 / 2)
        else:
            m = (ii - ci) ** 2 + (jj - cj) ** 2 <= s1 ** 2
        img[:, m] = val[:, None]
    if texture:
        img += 0.2 * (ii / H + jj / W)[None] / 2.0
        img += rng.uniform(-0.05, 0.05, size=img.shape)
    return np.clip(img, 0.0, 1.0)


def gaussian_kernel(K, sigma):
    r = (K - 1) / 2.0
    t = np.arange(K) - r
    g = np.exp(-(t[:, None] ** 2 + t[None, :] ** 2) / (2.0 * sigma ** 2))
    return g / g.sum()


def motion_kernel(K, length, angle_deg, samples=64):
    """Segment of the given length through the centre at the given angle
    (counter-clockwise from the +column axis, rows pointing down)."""
    r = (K - 1) / 2.0
    th = np.deg2rad(angle_deg)
    k = np.zeros((K, K))
    for s in np.linspace(-0.5, 0.5, samples):
        cj = r + s * (length - 1) * np.cos(th)
        ci = r - s * (length - 1) * np.sin(th)
        i0, j0 = int(np.floor(ci)), int(np.floor(cj))
        fi, fj = ci - i0, cj - j0
        for di, wi in ((0, 1 - fi), (1, fi)):
            for dj, wj in ((0, 1 - fj), (1, fj)):
                ii, jj = i0 + di, j0 + dj
                if 0 <= ii < K and 0 <= jj < K:
                    k[ii, jj] += wi * wj
    return k / k.sum()


def _periodic_blur(kernel, x):
    """Centred periodic convolution through the FFT (observation synthesis)."""
    C, H, W = x.shape
    K = kernel.shape[-1]
    r = (K - 1) // 2
    out = np.empty_like(x)
    for c in range(C):
        pad = np.zeros((H, W))
        for p in range(K):
            for q in range(K):
                pad[(p - r) % H, (q - r) % W] += kernel[c, p, q]
        out[c] = np.real(np.fft.ifft2(np.fft.fft2(pad) * np.fft.fft2(x[c])))
    return out


def _smooth_kernel_combine(k1, k2):
    """Full 2D convolution of two small kernels cropped to k1's size (used to
    build a motion-plus-Gaussian blur)."""
    K = k1.shape[0]
    full = np.zeros((2 * K - 1, 2 * K - 1))
    for p in range(k2.shape[0]):
        for q in range(k2.shape[1]):
            full[p:p + K, q:q + K] += k2[p, q] * k1
    o = (k2.shape[0] - 1) // 2
    out = full[o:o + K, o:o + K]
    return out / out.sum()


@dataclass
class Instance:
    """One deblurring instance: ground truth, observation and kernels."""
    name: str
    x_true: np.ndarray      # (C, H, W)
    y: np.ndarray           # (C, H, W) noisy blurred observation y^delta
    b_true: np.ndarray      # (C, K, K) kernel that generated y
    a: np.ndarray           # (C, K, K) kernel of A (and the initial b_0)
    noise: float
    params: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.x_true.shape

    @property
    def K(self):
        return self.a.shape[-1]


def make_instance(name, C, H, W, b_true, a, noise, seed, texture=True, **params):
    rng = np.random.default_rng(seed)
    x = piecewise_image(rng, C, H, W, texture=texture)
    bt = np.broadcast_to(b_true, (C,) + b_true.shape[-2:]).copy() if b_true.ndim == 2 else b_true
    aa = np.broadcast_to(a, (C,) + a.shape[-2:]).copy() if a.ndim == 2 else a
    y = _periodic_blur(bt, x) + noise * rng.standard_normal(x.shape)
    return Instance(name, x, y, bt, aa, noise, dict(params))


# ------------------------------------------------------------------ workloads

def gray64_k7(seed=0):
    """64 x 64 grayscale, true Gaussian sigma 1.5, initial sigma 1.0, noise 0.01,
    Huber 0.01, alpha 1e-2; run in float64."""
    return make_instance("gray64_k7_gauss_fp64", 1, 64, 64, gaussian_kernel(7, 1.5),
                         gaussian_kernel(7, 1.0), 0.01, seed, texture=False,
                         alpha=1e-2, reg_param=1e-2, beta=0.3, dtype="f64", upper_iters=50)


def rgb256_k15(seed=0):
    """256 x 256 RGB, 15 x 15 motion blur length 11 at 30 deg (shared across
    channels), initial kernel the same blur at 20 deg, noise 0.02."""
    return make_instance("rgb256_k15_motion", 3, 256, 256, motion_kernel(15, 11, 30),
                         motion_kernel(15, 11, 20), 0.02, seed,
                         alpha=1e-2, reg_param=1e-2, beta=0.3, dtype="f32")


def rgb512_k31(seed=0):
    """512 x 512 RGB, 31 x 31 Gaussian sigma 3 plus 10% positive perturbation,
    normalised; noise 0.01; the perturbed kernel is both A's kernel and b_0."""
    rng = np.random.default_rng(10_000 + seed)
    g = gaussian_kernel(31, 3.0)
    k = g + 0.1 * g.max() * rng.uniform(size=g.shape)
    k /= k.sum()
    return make_instance("rgb512_k31_gauss_perturbed", 3, 512, 512, k, k, 0.01, seed,
                         alpha=1e-2, reg_param=1e-2, beta=0.3, dtype="f32")


def rgb2048_k63(seed=0):
    """2048 x 2048 RGB, 63 x 63 motion (length 31 at 30 deg) convolved with a
    Gaussian sigma 3, noise 0.01."""
    k = _smooth_kernel_combine(motion_kernel(63, 31, 30), gaussian_kernel(19, 3.0))
    return make_instance("rgb2048_k63_motion_gauss", 3, 2048, 2048, k, k, 0.01, seed,
                         alpha=1e-2, reg_param=1e-2, beta=0.3, dtype="f32")


def diagonal_motion_kernel(K):
    """K x K motion blur along the main diagonal, equal weights summing to 1
    (the paper's 5 x 5 motion kernel of Sec. 4.2 has its non-zero entries on
    the diagonal; the weights are not given)."""
    return np.eye(K) / K


def paper2d_motion(seed=0):
    """The paper's 2D deblurring setting (Sec. 4.2) on a synthetic image:
    300 x 400 RGB, the 5 x 5 diagonal motion blur as the generating kernel, as
    A's kernel and as b_0, noise 0.02; sqrt-smoothed TV with nu = 1e-4,
    alpha 0.6, beta 0.3 on the H^1 seminorm (w0 = 0); run in float64 (the
    stop threshold is 1e-6)."""
    k = diagonal_motion_kernel(5)
    return make_instance("paper2d_motion", 3, 300, 400, k, k, 0.02, seed,
                         alpha=0.6, reg_param=1e-4, reg="sqrt", beta=0.3, w0=0.0, dtype="f64")


def paper2d_semiblind(seed=0):
    """Semi-blind variant of Sec. 4.2: the data is blurred by the motion kernel
    followed by a 5 x 5 Gaussian with sigma 0.5, and only the motion kernel is
    known (A's kernel and b_0).  The composed kernel is cropped to 5 x 5 and
    renormalised so that a 5 x 5 b can represent it."""
    km = diagonal_motion_kernel(5)
    kt = _smooth_kernel_combine(km, gaussian_kernel(5, 0.5))
    return make_instance("paper2d_semiblind", 3, 300, 400, kt, km, 0.02, seed,
                         alpha=0.6, reg_param=1e-4, reg="sqrt", beta=0.3, w0=0.0, dtype="f64")


def batch_mixed(n=64, seed=0, size_range=(128, 512), ks=(5, 9, 15, 21, 31)):
    """n independent RGB problems of uneven size and kernel (Gaussian or motion)."""
    rng = np.random.default_rng(20_000 + seed)
    out = []
    for i in range(n):
        s = int(rng.integers(size_range[0], size_range[1] + 1))
        K = int(rng.choice(ks))
        if rng.uniform() < 0.5:
            k = gaussian_kernel(K, rng.uniform(0.5, K / 6.0))
        else:
            k = motion_kernel(K, rng.uniform(3, K), rng.uniform(0, 180))
        out.append(make_instance(f"batch{i}", 3, s, s, k, k, float(rng.uniform(0.005, 0.03)),
                                 seed * 1000 + i, alpha=1e-2, reg_param=1e-2, beta=0.3,
                                 dtype="f32"))
    return out


def small(C=1, H=16, W=16, K=3, seed=0, noise=0.01, sigma_true=0.9, sigma_init=0.7,
          texture=False):
    """Tiny Gaussian-blur instance for oracle pins and quick parity checks."""
    return make_instance(f"small{C}x{H}x{W}k{K}", C, H, W, gaussian_kernel(K, sigma_true),
                         gaussian_kernel(K, sigma_init), noise, seed, texture=texture)


WORKLOADS = {
    "gray64_k7_gauss_fp64": gray64_k7,
    "rgb256_k15_motion": rgb256_k15,
    "rgb512_k31_gauss_perturbed": rgb512_k31,
    "rgb2048_k63_motion_gauss": rgb2048_k63,
    "paper2d_motion": paper2d_motion,
    "paper2d_semiblind": paper2d_semiblind,
}


@dataclass
class Signal1D:
    """A 1D deconvolution instance: the forward matrix A (also B_0), the signal
    and its noisy blurred observation."""
    name: str
    A: np.ndarray
    x_true: np.ndarray
    y: np.ndarray
    params: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.x_true.shape[0]


def gaussian_conv_matrix(n, sigma=5.0, cut=3.0):
    """A[t, tau] = k(t - tau) for the Gaussian k of std sigma on |d| <= cut
    sigma, normalised to sum 1; zero outside the signal."""
    r = int(np.ceil(cut * sigma))
    d = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (d / sigma) ** 2)
    k /= k.sum()
    A = np.zeros((n, n))
    t = np.arange(n)
    for j, dd in enumerate(range(-r, r + 1)):
        tau = t - dd
        ok = (tau >= 0) & (tau < n)
        A[t[ok], tau[ok]] = k[j]
    return A


def signal1d(n=256, seed=0, noise=5e-3, sigma=5.0):
    """Sec. 4.1's 1D setting on a synthetic sparse, piecewise-constant signal
    (the paper's own signal is not available): elastic net with
    a1 = 1.2e-3, a2 = 4e-3, proximal-gradient step 0.1, beta = 0."""
    rng = np.random.default_rng(30_000 + seed)
    x = np.zeros(n)
    for _ in range(max(3, n // 32)):
        L = int(rng.integers(max(1, n // 32), max(2, n // 8) + 1))
        s0 = int(rng.integers(0, max(1, n - L)))
        x[s0:s0 + L] = rng.uniform(0.2, 1.0)
    for _ in range(max(2, n // 64)):
        x[int(rng.integers(0, n))] = rng.uniform(0.3, 1.0)
    A = gaussian_conv_matrix(n, sigma)
    y = A @ x + noise * rng.standard_normal(n)
    return Signal1D(f"signal1d_n{n}", A, x, y, dict(a1=1.2e-3, a2=4e-3, lam=0.1, noise=noise))
