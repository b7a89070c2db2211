"""Seeded synthetic inputs: leaf Gaussians, camera paths and target images.

This module is the only code shared by the CUDA path's tests/bench and the CPU
oracle.  It holds none of the method's arithmetic (no hierarchy, selection,
projection or blending): it only draws random numbers and lays them out.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-based: value `i`
of stream `(seed, stream)` is `mix(key + (i + 1) * GOLDEN)` with
`key = mix(seed * 2**32 + stream)`, where `mix` is the SplitMix64 output
function.  Uniforms take the top 24 bits (exact in float32); normals use the
Box-Muller transform in float64.

Leaf record layout (float32, one row per Gaussian, row stride padded to a
multiple of 8 floats = 32 bytes):
  [0:3] mean mu, [3:6] scales s (linear), [6:10] rotation quaternion (w,x,y,z),
  [10] opacity sigma in [0,1], [11:14] base colour b (RGB),
  [14:14+3K] SH coefficients f for degrees 1..D, coefficient-major, RGB-minor,
  K = (D+1)^2 - 1 (the paper's count excludes the DC term; Sec. 3, 3DGS
  preliminaries).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

REC_MU, REC_S, REC_Q, REC_OP, REC_B, REC_F = 0, 3, 6, 10, 11, 14


def sh_coeff_count(degree: int) -> int:
    """Number of SH coefficients per channel excluding DC: (D+1)^2 - 1."""
    return (degree + 1) * (degree + 1) - 1


def record_stride(degree: int) -> int:
    """Floats per record row: 14 + 3K rounded up to a multiple of 8."""
    k = 14 + 3 * sh_coeff_count(degree)
    return (k + 7) // 8 * 8


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def hash_u64(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64: the (idx+1)-th output of stream (seed, stream)."""
    key = _mix(np.array([(seed << 32) + stream], dtype=np.uint64))[0]
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + (idx + np.uint64(1)) * GOLDEN)


def uniform(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """U[0,1) with 24 random bits (float64, exactly representable in float32)."""
    return (hash_u64(seed, stream, idx) >> np.uint64(40)).astype(np.float64) * (1.0 / 16777216.0)


def uniform_open(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """U(0,1) strictly inside, for logarithms."""
    return ((hash_u64(seed, stream, idx) >> np.uint64(40)).astype(np.float64) + 0.5) * (1.0 / 16777216.0)


def normal(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Standard normal by Box-Muller from two uniform streams (2*stream, 2*stream+1) + 1e6."""
    u1 = uniform_open(seed, 1_000_000 + 2 * stream, idx)
    u2 = uniform(seed, 1_000_000 + 2 * stream + 1, idx)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------------------
# leaves
# ---------------------------------------------------------------------------

def _common_attributes(rec: np.ndarray, seed: int, idx: np.ndarray, degree: int,
                       log_scale_mu: float, log_scale_sigma: float,
                       sh_sigma: float) -> None:
    for a in range(3):
        rec[:, REC_S + a] = np.exp(log_scale_mu + log_scale_sigma * normal(seed, 10 + a, idx))
    q = np.stack([normal(seed, 20 + a, idx) for a in range(4)], axis=1)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    rec[:, REC_Q:REC_Q + 4] = q
    rec[:, REC_OP] = 0.1 + 0.8 * uniform(seed, 30, idx)
    for c in range(3):
        rec[:, REC_B + c] = uniform(seed, 31 + c, idx)
    nf = 3 * sh_coeff_count(degree)
    for k in range(nf):
        rec[:, REC_F + k] = sh_sigma * normal(seed, 40 + k, idx)


def leaves_uniform_cube(n: int, seed: int, half_extent: float = 50.0, degree: int = 0,
                        log_scale_mu: float = -1.0, log_scale_sigma: float = 0.5,
                        sh_sigma: float = 0.2) -> np.ndarray:
    """Means uniform in [-h,h]^3, log-normal scales, random unit quaternions,
    opacity U[0.1,0.9], base colour U[0,1]^3, SH ~ N(0, sh_sigma^2)."""
    idx = np.arange(n, dtype=np.uint64)
    rec = np.zeros((n, record_stride(degree)), dtype=np.float64)
    for a in range(3):
        rec[:, REC_MU + a] = -half_extent + 2.0 * half_extent * uniform(seed, a, idx)
    _common_attributes(rec, seed, idx, degree, log_scale_mu, log_scale_sigma, sh_sigma)
    return rec.astype(np.float32)


def leaves_ground_and_boxes(n: int, seed: int, degree: int = 3, extent: float = 1000.0,
                            ground_frac: float = 0.7, n_boxes: int = 256,
                            log_scale_mu: float = -1.0, log_scale_sigma: float = 0.5,
                            sh_sigma: float = 0.2) -> np.ndarray:
    """Clustered density, world z up: `ground_frac` of the leaves on a square
    ground plane of side `extent` (z jitter N(0, 0.05^2)), the rest uniform
    inside `n_boxes` boxes (footprint U[10,40] m, height U[5,60] m, centres
    uniform on the plane)."""
    idx = np.arange(n, dtype=np.uint64)
    rec = np.zeros((n, record_stride(degree)), dtype=np.float64)
    h = 0.5 * extent
    n_ground = int(round(ground_frac * n))
    g = idx[:n_ground]
    rec[:n_ground, 0] = -h + extent * uniform(seed, 0, g)
    rec[:n_ground, 1] = -h + extent * uniform(seed, 1, g)
    rec[:n_ground, 2] = 0.05 * normal(seed, 2, g)
    bidx = np.arange(n_boxes, dtype=np.uint64)
    bcx = -h + extent * uniform(seed, 100, bidx)
    bcy = -h + extent * uniform(seed, 101, bidx)
    bwx = 10.0 + 30.0 * uniform(seed, 102, bidx)
    bwy = 10.0 + 30.0 * uniform(seed, 103, bidx)
    bh = 5.0 + 55.0 * uniform(seed, 104, bidx)
    b = idx[n_ground:]
    box = np.minimum((uniform(seed, 3, b) * n_boxes).astype(np.int64), n_boxes - 1)
    rec[n_ground:, 0] = bcx[box] + bwx[box] * (uniform(seed, 4, b) - 0.5)
    rec[n_ground:, 1] = bcy[box] + bwy[box] * (uniform(seed, 5, b) - 0.5)
    rec[n_ground:, 2] = bh[box] * uniform(seed, 6, b)
    _common_attributes(rec, seed, idx, degree, log_scale_mu, log_scale_sigma, sh_sigma)
    return rec.astype(np.float32)


# ---------------------------------------------------------------------------
# cameras
# ---------------------------------------------------------------------------

@dataclass
class Camera:
    """Pinhole camera.  R is world->camera (rows: right, down, forward), pos is
    the camera centre in world coordinates; +z forward, +x right, +y down."""
    R: np.ndarray
    pos: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    tau: float = 1.0
    znear: float = 0.2
    spt_scale: float = 1.0        # factor on the SPT root distances (training LoD noise)
    extra: dict = field(default_factory=dict)


def lod_noise_factor(r: float) -> float:
    """LoD noise of training: distances to the SPT roots are multiplied by 1 + 5 r^4,
    r ~ U(0, 1) drawn once per iteration (appendix "Varying level of detail")."""
    return 1.0 + 5.0 * float(r) ** 4


def camera_look(pos, forward, right, width: int, height: int, fovx_deg: float = 60.0,
                tau: float = 1.0, znear: float = 0.2) -> Camera:
    f = np.asarray(forward, dtype=np.float64)
    f /= np.linalg.norm(f)
    r = np.asarray(right, dtype=np.float64)
    r = r - f * np.dot(r, f)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f], axis=0).astype(np.float32)
    fx = (0.5 * width) / math.tan(math.radians(0.5 * fovx_deg))
    return Camera(R=R, pos=np.asarray(pos, dtype=np.float32), fx=np.float32(fx), fy=np.float32(fx),
                  cx=np.float32(0.5 * width), cy=np.float32(0.5 * height), width=width,
                  height=height, tau=np.float32(tau), znear=np.float32(znear))


def aerial_to_street_path(n_views: int = 32, width: int = 1920, height: int = 1080,
                          alt_hi: float = 500.0, alt_lo: float = 2.0, travel: float = 600.0,
                          tau: float = 1.0) -> list[Camera]:
    """Altitude geometric alt_hi -> alt_lo, pitch -90 deg -> -5 deg, the looked-at
    ground point moving linearly across `travel` metres along +x (world z up)."""
    cams = []
    for v in range(n_views):
        t = v / max(1, n_views - 1)
        alt = alt_hi * (alt_lo / alt_hi) ** t
        pitch = math.radians(-90.0 + 85.0 * t)
        fwd = np.array([math.cos(pitch), 0.0, math.sin(pitch)])
        g = np.array([-0.5 * travel + travel * t, 0.0, 0.0])
        pos = g - fwd * (alt / -math.sin(pitch))
        cams.append(camera_look(pos, fwd, [0.0, -1.0, 0.0], width, height, tau=tau))
    return cams


def target_image(seed: int, height: int, width: int) -> np.ndarray:
    """Seeded U[0,1) target image, HWC float32."""
    idx = np.arange(height * width * 3, dtype=np.uint64)
    return uniform(seed, 7, idx).astype(np.float32).reshape(height, width, 3)


def target_bytes(seed: int, height: int, width: int) -> np.ndarray:
    """Seeded 8-bit RGB target image (bytes uniform on 0..255), HWC uint8."""
    idx = np.arange(height * width * 3, dtype=np.uint64)
    return np.minimum(np.floor(uniform(seed, 8, idx) * 256.0), 255.0).astype(np.uint8).reshape(height, width, 3)


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

def config1_scene() -> dict:
    """65,536 leaves in a 100 m cube, SH degree 0; one 256x256 camera at 60 deg."""
    leaves = leaves_uniform_cube(65536, seed=1, degree=0)
    cam = camera_look([0.0, 0.0, -120.0], [0.0, 0.0, 1.0], [1.0, 0.0, 0.0], 256, 256, tau=1.0)
    return {"leaves": leaves, "degree": 0, "cameras": [cam], "spt_volume": 700.0,
            "kappa": float(cam.fx / cam.tau)}


def config2_scene(n: int = 2_097_152, n_views: int = 32, width: int = 1920, height: int = 1080) -> dict:
    """2M leaves, SH degree 3, 70% ground / 30% boxes; aerial-to-street path at 1080p."""
    leaves = leaves_ground_and_boxes(n, seed=2, degree=3)
    cams = aerial_to_street_path(n_views, width, height)
    return {"leaves": leaves, "degree": 3, "cameras": cams, "spt_volume": 400.0,
            "kappa": float(cams[0].fx / cams[0].tau)}


# ---------------------------------------------------------------------------
# device-side generation for the large scenes (same hash, torch int64 lanes)
# ---------------------------------------------------------------------------

def _to_i64(u: int) -> int:
    return u - (1 << 64) if u >= (1 << 63) else u


_GOLDEN_I = _to_i64(0x9E3779B97F4A7C15)
_M1_I = _to_i64(0xBF58476D1CE4E5B9)
_M2_I = _to_i64(0x94D049BB133111EB)


def _srl(z, k: int):
    """Logical right shift of int64 lanes holding uint64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix_t(z):
    z = (z ^ _srl(z, 30)) * _M1_I
    z = (z ^ _srl(z, 27)) * _M2_I
    return z ^ _srl(z, 31)


def hash_u64_t(seed: int, stream: int, idx):
    """Torch version of hash_u64 (bit-identical), idx an int64 tensor."""
    key = int(_mix(np.array([(seed << 32) + stream], dtype=np.uint64))[0])
    return _mix_t(_to_i64(key) + (idx + 1) * _GOLDEN_I)


def uniform_t(seed: int, stream: int, idx):
    import torch
    return _srl(hash_u64_t(seed, stream, idx), 40).to(torch.float64) * (1.0 / 16777216.0)


def normal_t(seed: int, stream: int, idx):
    import torch
    u1 = (_srl(hash_u64_t(seed, 1_000_000 + 2 * stream, idx), 40).to(torch.float64) + 0.5) * (1.0 / 16777216.0)
    u2 = uniform_t(seed, 1_000_000 + 2 * stream + 1, idx)
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)


def city_leaves_t(n: int, seed: int, degree: int = 3, extent: float = 2000.0, block: float = 100.0,
                  ground_frac: float = 0.4, device: str = "cuda", chunk: int = 1 << 22,
                  log_scale_mu: float = -1.0, log_scale_sigma: float = 0.5, sh_sigma: float = 0.2):
    """City-like leaves generated on the device: a square street grid of
    `block`-metre blocks, one box building per block (footprint U[30,70] m,
    height U[10,120] m); `ground_frac` of the leaves on the ground (z jitter
    N(0, 0.05^2)), the rest uniform on building walls and roofs (face chosen by
    area).  Attributes as in leaves_uniform_cube.  Returns an n x stride
    float32 tensor on `device`."""
    import torch
    st = record_stride(degree)
    out = torch.zeros((n, st), dtype=torch.float32, device=device)
    nb = int(extent // block)
    bidx = torch.arange(nb * nb, dtype=torch.int64, device=device)
    bw = 30.0 + 40.0 * uniform_t(seed, 200, bidx)
    bd = 30.0 + 40.0 * uniform_t(seed, 201, bidx)
    bh = 10.0 + 110.0 * uniform_t(seed, 202, bidx)
    bcx = -0.5 * extent + block * (torch.remainder(bidx, nb).to(torch.float64) + 0.5)
    bcy = -0.5 * extent + block * (torch.div(bidx, nb, rounding_mode="floor").to(torch.float64) + 0.5)
    areas = torch.stack([bw * bh, bw * bh, bd * bh, bd * bh, bw * bd], dim=1)
    cum = torch.cumsum(areas, dim=1)
    cum = cum / cum[:, -1:]
    n_ground = int(round(ground_frac * n))
    K = sh_coeff_count(degree)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        i = torch.arange(s, e, dtype=torch.int64, device=device)
        pos = torch.zeros((e - s, 3), dtype=torch.float64, device=device)
        g = i < n_ground
        ux, uy = uniform_t(seed, 0, i), uniform_t(seed, 1, i)
        pos[:, 0] = -0.5 * extent + extent * ux
        pos[:, 1] = -0.5 * extent + extent * uy
        pos[:, 2] = 0.05 * normal_t(seed, 2, i)
        b = torch.clamp((uniform_t(seed, 3, i) * (nb * nb)).to(torch.int64), max=nb * nb - 1)
        f = torch.searchsorted(cum[b], uniform_t(seed, 4, i).unsqueeze(1)).squeeze(1).clamp(max=4)
        a, c = uniform_t(seed, 5, i) - 0.5, uniform_t(seed, 6, i)
        hx, hy = 0.5 * bw[b], 0.5 * bd[b]
        wx = torch.where(f <= 1, a * bw[b], torch.where(f == 2, -hx, torch.where(f == 3, hx, a * bw[b])))
        wy = torch.where(f == 0, -hy, torch.where(f == 1, hy, torch.where(f <= 3, a * bd[b], (c - 0.5) * bd[b])))
        wz = torch.where(f == 4, bh[b], c * bh[b])
        bpos = torch.stack([bcx[b] + wx, bcy[b] + wy, wz], dim=1)
        pos = torch.where(g.unsqueeze(1), pos, bpos)
        rec = out[s:e]
        rec[:, 0:3] = pos.to(torch.float32)
        for k in range(3):
            rec[:, REC_S + k] = torch.exp(log_scale_mu + log_scale_sigma * normal_t(seed, 10 + k, i)).float()
        q = torch.stack([normal_t(seed, 20 + k, i) for k in range(4)], dim=1)
        q = q / torch.linalg.norm(q, dim=1, keepdim=True)
        rec[:, REC_Q:REC_Q + 4] = q.float()
        rec[:, REC_OP] = (0.1 + 0.8 * uniform_t(seed, 30, i)).float()
        for c3 in range(3):
            rec[:, REC_B + c3] = uniform_t(seed, 31 + c3, i).float()
        for k in range(3 * K):
            rec[:, REC_F + k] = (sh_sigma * normal_t(seed, 40 + k, i)).float()
    return out


def flyover_path(n: int = 40, width: int = 320, height: int = 180) -> list[Camera]:
    """A slow pass over the 300 m ground-and-boxes scene at altitude 35 -> 25 m,
    looking forward and down; the view distance changes by under a percent a
    view."""
    cams = []
    for i in range(n):
        s = i / (n - 1)
        pos = [-100.0 + 200.0 * s, -60.0, 35.0 - 10.0 * s]
        cams.append(camera_look(pos, [0.3, 1.0, -0.7], [1.0, -0.3, 0.0], width, height, tau=1.0))
    return cams


def flythrough_path(n_views: int = 200, width: int = 1920, height: int = 1080, alt_hi: float = 300.0,
                    alt_lo: float = 20.0, tau: float = 1.0) -> list[Camera]:
    """Smooth flythrough: altitude geometric alt_hi -> alt_lo, pitch -60 deg ->
    -15 deg, heading turning through 90 degrees along a spiral; consecutive
    views move by well under 1% of the viewing distance."""
    cams = []
    for v in range(n_views):
        t = v / max(1, n_views - 1)
        alt = alt_hi * (alt_lo / alt_hi) ** t
        pitch = math.radians(-60.0 + 45.0 * t)
        head = math.radians(90.0 * t)
        r = 400.0 * (1.0 - 0.8 * t)
        pos = np.array([r * math.cos(head + math.pi), r * math.sin(head + math.pi), alt])
        fwd = np.array([math.cos(head) * math.cos(pitch), math.sin(head) * math.cos(pitch), math.sin(pitch)])
        right = np.array([math.sin(head), -math.cos(head), 0.0])
        cams.append(camera_look(pos, fwd, right, width, height, tau=tau))
    return cams


SERVING_RESOLUTIONS = ((640, 360), (1280, 720), (1920, 1080), (3840, 2160))
SERVING_TAUS = (0.5, 1.0, 2.0, 4.0)


def serving_cameras(n: int, seed: int, extent: float = 2000.0) -> list[Camera]:
    """Request cameras: resolution and LoD threshold uniform over the serving
    sets; half aerial (50-500 m, pitch -45..-90 deg), half street level
    (1.5-3 m, pitch -5..+5 deg), positions and headings uniform."""
    idx = np.arange(n, dtype=np.uint64)
    u = [uniform(seed, 600 + k, idx) for k in range(8)]
    cams = []
    for i in range(n):
        w, h = SERVING_RESOLUTIONS[int(u[0][i] * 4) % 4]
        tau = SERVING_TAUS[int(u[1][i] * 4) % 4]
        aerial = u[2][i] < 0.5
        x, y = (u[3][i] - 0.5) * 0.8 * extent, (u[4][i] - 0.5) * 0.8 * extent
        head = 2.0 * math.pi * u[5][i]
        if aerial:
            alt, pitch = 50.0 + 450.0 * u[6][i], math.radians(-45.0 - 44.0 * u[7][i])
        else:
            alt, pitch = 1.5 + 1.5 * u[6][i], math.radians(-5.0 + 10.0 * u[7][i])
        fwd = np.array([math.cos(head) * math.cos(pitch), math.sin(head) * math.cos(pitch), math.sin(pitch)])
        right = np.array([math.sin(head), -math.cos(head), 0.0])
        cams.append(camera_look([x, y, alt], fwd, right, w, h, tau=tau))
    return cams
