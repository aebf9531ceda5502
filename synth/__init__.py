"""Seeded synthetic inputs for rotational alignment (Gaussian-blob volumes).

This module only *makes inputs*.  It holds none of the alignment method's
arithmetic (no spherical harmonics, no Wigner functions, no correlation): the
oracle and the CUDA library both consume the float32 volumes it returns.

Recipe (one particle = one (template, particle) pair, each from its own seed):

* template ``h``: a sum of isotropic Gaussian blobs ``a*exp(-|x-c|^2/(2 sigma^2))``
  evaluated at voxel centres; blob centres uniform in a ball of the given
  radius around the box centre ``c0 = N/2`` (rejection sampling), amplitudes
  ``U[0.5, 1]``;
* ground truth rotation ``R*``: a normalised 4-vector of standard normals
  (a Haar-random unit quaternion);
* clean particle ``s(x) = h(R*^T (x - c0) + c0 - tau*)`` by trilinear
  interpolation of the template (or, with ``exact_rotation=True``, the blobs
  re-rendered at the centres ``R* (c - c0 + tau*) + c0``, which is the exact
  pose of a sum of isotropic Gaussians); the planted shift ``tau*`` is zero
  unless the workload sets ``shift_max`` (then uniform in a ball of that radius,
  in voxels), so that ``s = g* o S_tau* h`` with ``(S_tau h)(x) = h(x - tau)``;
* noise: i.i.d. Gaussian with variance ``mean_box(s^2) / SNR``;
* optional missing wedge (tilt axis y, beam z): keep the Fourier samples with
  ``|k_z| <= tan(wedge) * |k_x|`` plus the zero-frequency sample.

This stands in for the paper's particle model ``f = g* o h + noise``
(Section 5.1) on the subtomogram shapes of its experiments.  Volumes are C-order
``[z][y][x]``; voxel ``[k][j][i]`` sits at position ``(x, y, z) = (i, j, k)``.

Random draws come from ``numpy.random.SeedSequence(base_seed).spawn(B)``, one
child per particle, so results do not depend on the device that renders them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

__all__ = [
    "Workload", "WORKLOADS", "haar_rotation", "blob_params", "render_blobs",
    "rotate_trilinear", "apply_missing_wedge", "make_batch",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """A synthetic workload: volume recipe plus the alignment parameters."""
    name: str
    B: int
    N: int
    n_blobs: int
    sigma: float
    ball_radius: float
    snr: float
    wedge_deg: Optional[float]
    n_shells: int
    L_sched: Sequence[int]
    L0: int
    K: int
    P: int
    M_iter: int
    base_seed: int
    shared_template: bool = False
    snr_range: Optional[Tuple[float, float]] = None  # per-particle SNR ~ U[lo, hi] (overrides snr)
    P_range: Optional[Tuple[int, int]] = None        # per-particle candidate count ~ U{lo..hi}
    seed_offset: int = 0                             # index of particle 0 in the seed sequence
    shift_max: float = 0.0                           # planted shift tau* uniform in this ball (voxels)
    rounds: int = 1                                  # rotation-translation alternations (6-D pose)
    max_shift: int = 0                               # integer shift search window, voxels per axis

    @property
    def r_max(self) -> float:
        return self.N / 2 - 1.0

    @property
    def L_final(self) -> int:
        return int(self.L_sched[-1])


# The two single-GPU workloads: a small FP64 case the oracle finishes in
# seconds, and the 1024-particle 64^3 batch the throughput metric is quoted on.
WORKLOADS = {
    "small32": Workload("small32", B=1, N=32, n_blobs=16, sigma=1.5, ball_radius=12.0,
                        snr=0.5, wedge_deg=None, n_shells=12, L_sched=(8, 12, 16),
                        L0=8, K=2, P=8, M_iter=3, base_seed=20260316),
    "batch64": Workload("batch64", B=1024, N=64, n_blobs=48, sigma=2.0, ball_radius=26.0,
                        snr=0.1, wedge_deg=60.0, n_shells=32, L_sched=(8, 16, 24, 32),
                        L0=8, K=2, P=16, M_iter=3, base_seed=20260317),
    "deep64": Workload("deep64", B=2048, N=64, n_blobs=48, sigma=2.0, ball_radius=26.0,
                       snr=0.1, wedge_deg=60.0, n_shells=32, L_sched=(8, 16, 24, 32, 40, 48),
                       L0=8, K=2, P=16, M_iter=3, base_seed=20260319),
    # A batch mixing box sizes (2048 x 48^3, 1024 x 64^3, 1024 x 96^3 items of one
    # seed sequence, in that order): per-particle SNR ~ U[0.05, 0.3] and candidate
    # count ~ U{8..32}, blobs in a ball of radius floor(0.4 N), S = final L shells.
    "var48": Workload("var48", B=2048, N=48, n_blobs=32, sigma=2.0, ball_radius=19.0,
                      snr=None, wedge_deg=60.0, n_shells=24, L_sched=(8, 16, 24),
                      L0=8, K=2, P=32, M_iter=3, base_seed=20260318, snr_range=(0.05, 0.3),
                      P_range=(8, 32), seed_offset=0),
    "var64": Workload("var64", B=1024, N=64, n_blobs=48, sigma=2.0, ball_radius=25.0,
                      snr=None, wedge_deg=60.0, n_shells=32, L_sched=(8, 16, 24, 32),
                      L0=8, K=2, P=32, M_iter=3, base_seed=20260318, snr_range=(0.05, 0.3),
                      P_range=(8, 32), seed_offset=2048),
    "var96": Workload("var96", B=1024, N=96, n_blobs=96, sigma=2.0, ball_radius=38.0,
                      snr=None, wedge_deg=60.0, n_shells=48, L_sched=(8, 16, 24, 32, 40, 48),
                      L0=8, K=2, P=32, M_iter=3, base_seed=20260318, snr_range=(0.05, 0.3),
                      P_range=(8, 32), seed_offset=3072),
    "grad64": Workload("grad64", B=512, N=64, n_blobs=48, sigma=2.0, ball_radius=26.0,
                       snr=0.2, wedge_deg=60.0, n_shells=32, L_sched=(8, 16, 24, 32),
                       L0=8, K=2, P=16, M_iter=3, base_seed=20260320, shared_template=True),
    # The largest bandwidth the library takes (L_J = 64), a short batch.
    "max64": Workload("max64", B=8, N=64, n_blobs=48, sigma=2.0, ball_radius=26.0,
                      snr=0.1, wedge_deg=60.0, n_shells=32, L_sched=(8, 16, 32, 64),
                      L0=8, K=2, P=16, M_iter=3, base_seed=20260322),
    # The paper's own regime: 200^3 boxes, SOFFT at L0 = 30 with K = 2 (a 124^3
    # grid), P = 10 candidates, one Newton step per band, final L = 40, at 0 dB.
    "paper200": Workload("paper200", B=256, N=200, n_blobs=160, sigma=3.0, ball_radius=80.0,
                         snr=1.0, wedge_deg=60.0, n_shells=40, L_sched=(30, 40),
                         L0=30, K=2, P=10, M_iter=1, base_seed=20260321),
    # Bandwidths above 64 (up to the paper's L_max <= 100): a 64^3 pair marched to
    # L = 100, and the paper's own schedules at 200^3: {30, 40, 60, 100} with one
    # Newton step per band, and M_iter = 5 over {30, 40, 45} (its STA setting).
    "wide64": Workload("wide64", B=2, N=64, n_blobs=48, sigma=2.0, ball_radius=26.0,
                       snr=0.1, wedge_deg=60.0, n_shells=32, L_sched=(8, 16, 32, 64, 100),
                       L0=8, K=2, P=8, M_iter=3, base_seed=20260325),
    "paper200w": Workload("paper200w", B=4, N=200, n_blobs=160, sigma=3.0, ball_radius=80.0,
                          snr=1.0, wedge_deg=60.0, n_shells=40, L_sched=(30, 40, 60, 100),
                          L0=30, K=2, P=10, M_iter=1, base_seed=20260321),
    "sta200": Workload("sta200", B=4, N=200, n_blobs=160, sigma=3.0, ball_radius=80.0,
                       snr=1.0, wedge_deg=60.0, n_shells=40, L_sched=(30, 40, 45),
                       L0=30, K=2, P=10, M_iter=5, base_seed=20260321),
    # 6-D pose (rotation and translation): planted shifts up to 3 voxels, three
    # rotation-translation alternations, integer search window +-5 voxels.
    "shift32": Workload("shift32", B=2, N=32, n_blobs=16, sigma=1.5, ball_radius=10.0,
                        snr=0.5, wedge_deg=None, n_shells=12, L_sched=(8, 12, 16),
                        L0=8, K=2, P=8, M_iter=3, base_seed=20260323, shift_max=2.5,
                        rounds=3, max_shift=4),
    "shift64": Workload("shift64", B=1024, N=64, n_blobs=48, sigma=2.0, ball_radius=24.0,
                        snr=0.1, wedge_deg=60.0, n_shells=32, L_sched=(8, 16, 24, 32),
                        L0=8, K=2, P=16, M_iter=3, base_seed=20260324, shift_max=3.0,
                        rounds=3, max_shift=5),
}


def haar_rotation(rng: np.random.Generator) -> np.ndarray:
    """Haar-random rotation matrix from a normalised Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def blob_params(rng: np.random.Generator, n_blobs: int, ball_radius: float):
    """Blob centre offsets (uniform in a ball, rejection sampled) and amplitudes."""
    cs = []
    while len(cs) < n_blobs:
        p = rng.uniform(-ball_radius, ball_radius, size=3)
        if p @ p <= ball_radius * ball_radius:
            cs.append(p)
    amps = rng.uniform(0.5, 1.0, size=n_blobs)
    return np.array(cs), amps


def render_blobs(N: int, offsets, amps, sigma: float, device="cpu") -> torch.Tensor:
    """Sum of isotropic Gaussians at voxel centres; float64 [z][y][x].

    ``offsets`` [n][3] (x, y, z relative to N/2) and ``amps`` [n], or batched
    [B][n][3] and [B][n] for a [B][z][y][x] result.  An isotropic Gaussian
    factorises over x, y, z, so each volume is a sum of outer products of
    three 1-D profiles.
    """
    c0 = N / 2
    grid = torch.arange(N, dtype=torch.float64, device=device) - c0
    off = torch.as_tensor(offsets, dtype=torch.float64, device=device)
    a = torch.as_tensor(amps, dtype=torch.float64, device=device)
    batched = off.dim() == 3
    if not batched:
        off, a = off[None], a[None]
    g = torch.exp(-(grid[None, None, None, :] - off[..., None]) ** 2 / (2 * sigma * sigma))  # [B][n][xyz][N]
    v = torch.einsum("cb,cbz,cby,cbx->czyx", a, g[:, :, 2], g[:, :, 1], g[:, :, 0])
    return v if batched else v[0]


def rotate_trilinear(vol: torch.Tensor, R, shift=None) -> torch.Tensor:
    """out(x) = vol(R^T (x - c0) + c0 - shift) by trilinear interpolation, zero outside.

    ``vol`` [N][N][N] with R [3][3] (shift [3] or None), or batched
    [B][N][N][N] with R [B][3][3] (shift [B][3] or None).
    """
    batched = vol.dim() == 4
    if not batched:
        vol, R = vol[None], np.asarray(R)[None]
        shift = None if shift is None else np.asarray(shift)[None]
    Bn, N = vol.shape[0], vol.shape[-1]
    dev = vol.device
    c0 = N / 2
    Rt = torch.as_tensor(np.asarray(R), dtype=torch.float64, device=dev)   # [B][3][3]
    ax = torch.arange(N, dtype=torch.float64, device=dev) - c0
    zz, yy, xx = torch.meshgrid(ax, ax, ax, indexing="ij")
    x = torch.stack([xx, yy, zz], -1).reshape(-1, 3)                          # [V][3]
    pts = torch.einsum("vj,bij->bvi", x, Rt.transpose(1, 2)) + c0             # R^T x + c0
    if shift is not None:
        pts = pts - torch.as_tensor(np.asarray(shift), dtype=torch.float64, device=dev)[:, None, :]
    i0 = torch.floor(pts).long()
    fr = pts - i0
    out = torch.zeros(pts.shape[:2], dtype=vol.dtype, device=dev)
    flat = vol.reshape(Bn, -1)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                ix, iy, iz = i0[..., 0] + dx, i0[..., 1] + dy, i0[..., 2] + dz
                w = ((fr[..., 0] if dx else 1 - fr[..., 0]) * (fr[..., 1] if dy else 1 - fr[..., 1])
                     * (fr[..., 2] if dz else 1 - fr[..., 2]))
                ok = (ix >= 0) & (ix < N) & (iy >= 0) & (iy < N) & (iz >= 0) & (iz < N)
                lin = (iz.clamp(0, N - 1) * N + iy.clamp(0, N - 1)) * N + ix.clamp(0, N - 1)
                out += torch.where(ok, w * torch.gather(flat, 1, lin), torch.zeros_like(w))
    out = out.reshape(Bn, N, N, N)
    return out if batched else out[0]


def apply_missing_wedge(vol: torch.Tensor, wedge_deg: float) -> torch.Tensor:
    """Zero the Fourier samples outside a +-wedge_deg tilt range (axis y, beam z).

    Acts on the last three axes, so batches of volumes work unchanged.
    """
    N = vol.shape[-1]
    F = torch.fft.fftn(vol, dim=(-3, -2, -1))
    k = torch.fft.fftfreq(N, device=vol.device, dtype=torch.float64)
    kz, ky, kx = torch.meshgrid(k, k, k, indexing="ij")
    keep = kz.abs() <= math.tan(math.radians(wedge_deg)) * kx.abs() + 1e-12
    keep |= (kz == 0) & (kx == 0) & (ky == 0)
    return torch.fft.ifftn(F * keep, dim=(-3, -2, -1)).real


def make_batch(w: Workload, B: Optional[int] = None, start: int = 0, device="cpu",
               exact_rotation: bool = False, noise: bool = True, chunk: int = 64):
    """Generate particles ``start .. start+B-1`` of workload ``w``.

    Returns dict with ``templates`` (float32 [Bt][N][N][N], Bt = 1 when the
    workload shares one template, else B), ``particles`` (float32 [B][N][N][N]),
    ``R_true`` (float64 [B][3][3]), ``tau_true`` (float64 [B][3], (x, y, z)
    voxels; zero unless the workload plants shifts).  Random draws are made per particle on the
    host; rendering runs in chunks of ``chunk`` particles on ``device``.
    """
    B = w.B if B is None else B
    first = w.seed_offset + start
    seeds = np.random.SeedSequence(w.base_seed).spawn(first + B)[first:]
    N = w.N
    parts = torch.empty((B, N, N, N), dtype=torch.float32, device=device)
    temps = None if w.shared_template else torch.empty((B, N, N, N), dtype=torch.float32, device=device)
    Rs = np.empty((B, 3, 3))
    taus = np.zeros((B, 3))
    snrs = np.full(B, w.snr if w.snr is not None else 0.0)
    P_per = np.full(B, w.P, dtype=np.int32)
    shared = None
    if w.shared_template:
        trng = np.random.default_rng(np.random.SeedSequence(w.base_seed + 7919))
        offs, amps = blob_params(trng, w.n_blobs, w.ball_radius)
        shared = (offs, amps, render_blobs(N, offs, amps, w.sigma, device))
        temps = shared[2].float()[None].contiguous()
    for c0 in range(0, B, chunk):
        idx = range(c0, min(B, c0 + chunk))
        offs_l, amps_l, etas = [], [], []
        for b in idx:
            rng = np.random.default_rng(seeds[b])
            if shared is None:
                offs, amps = blob_params(rng, w.n_blobs, w.ball_radius)
            else:
                offs, amps = shared[0], shared[1]
            offs_l.append(offs); amps_l.append(amps)
            Rs[b] = haar_rotation(rng)
            if w.snr_range is not None:
                snrs[b] = rng.uniform(*w.snr_range)
            if w.P_range is not None:
                P_per[b] = rng.integers(w.P_range[0], w.P_range[1] + 1)
            if w.shift_max > 0:
                while True:
                    t = rng.uniform(-w.shift_max, w.shift_max, size=3)
                    if t @ t <= w.shift_max * w.shift_max:
                        break
                taus[b] = t
            if noise and snrs[b] > 0:
                etas.append(rng.standard_normal((N, N, N), dtype=np.float32))
        Rc = Rs[c0:c0 + len(idx)]
        tc = taus[c0:c0 + len(idx)] if w.shift_max > 0 else None
        if shared is None:
            h = render_blobs(N, np.stack(offs_l), np.stack(amps_l), w.sigma, device)
            temps[c0:c0 + len(idx)] = h.float()
        else:
            h = shared[2][None].expand(len(idx), N, N, N)
        if exact_rotation:
            o = np.stack(offs_l) + (0.0 if tc is None else tc[:, None, :])
            rot = np.einsum("bnj,bij->bni", o, Rc)
            s = render_blobs(N, rot, np.stack(amps_l), w.sigma, device)
        else:
            s = rotate_trilinear(h.contiguous(), Rc, tc)
        if etas:
            snr = torch.as_tensor(snrs[c0:c0 + len(idx)], dtype=s.dtype, device=device)
            var = (s * s).mean(dim=(1, 2, 3)) / snr
            eta = torch.from_numpy(np.stack(etas)).to(device=device, dtype=s.dtype)
            s = s + var.sqrt()[:, None, None, None] * eta
        if w.wedge_deg is not None:
            s = apply_missing_wedge(s, w.wedge_deg)
        parts[c0:c0 + len(idx)] = s.float()
    return {
        "templates": temps,
        "particles": parts,
        "R_true": Rs,
        "tau_true": taus,
        "snr": snrs,
        "P_per": P_per,
    }
