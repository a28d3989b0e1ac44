"""Seeded synthetic inputs shared by the CUDA path, its tests, the bench and the oracle.

This module draws random numbers and lays out configuration data. It holds none of the
method's arithmetic: no frustum construction, no froxelization, no network, no loss.
Everything random that the method consumes (scene boxes, viewcells, ground-truth sample
points, initial weights) is drawn here and passed in as plain arrays.

Random numbers: SplitMix64 (Steele, Lea, Flood 2014), used as a counter-based generator:
output i of a stream with seed S is mix(S + (i+1) * 0x9E3779B97F4A7C15), with
mix(z) = z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27; z *= 0x94D049BB133111EB; z ^= z>>31.
A uniform double is (u64 >> 11) * 2^-53. A normal is Box-Muller on two uniforms. Each purpose
uses its own stream, whose seed is mix(seed * 0x100000001B3 + stream_id + 1).

Workload shapes follow the paper's setting (froxel grids in a view frustum, Sec. 3.1-3.2;
interleave factor d, Sec. 3.3; viewcells with FOV 60 deg widened by 2x15 deg, Sec. 4.3).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1

# stream ids (purposes)
STREAM_SCENE = 1
STREAM_VIEWCELL = 2
STREAM_WEIGHTS = 3
STREAM_GT_POINTS = 4
STREAM_MISC = 5


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * _M1
        z = z ^ (z >> np.uint64(27))
        z = z * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _mix_int(z: int) -> int:
    return int(_mix(np.array([z & _MASK], dtype=np.uint64))[0])


def stream_seed(seed: int, stream: int) -> int:
    return _mix_int((seed * 0x100000001B3 + stream + 1) & _MASK)


class Rng:
    """Counter-based SplitMix64 stream."""

    def __init__(self, seed: int, stream: int = 0):
        self.seed = stream_seed(seed, stream)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            z = np.uint64(self.seed) + idx * _GAMMA
        return _mix(z)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        u = self.uniform(2 * n).reshape(n, 2)
        return np.sqrt(-2.0 * np.log1p(-u[:, 0])) * np.cos(2.0 * math.pi * u[:, 1])


# ----------------------------------------------------------------------------------------------
# Scenes: axis-aligned boxes, float32 [n][6] = (minx, miny, minz, maxx, maxy, maxz)
# ----------------------------------------------------------------------------------------------

def random_boxes(seed: int = 0, n: int = 40, world=(100.0, 20.0, 100.0), ext=(1.0, 8.0)) -> np.ndarray:
    """n boxes, centres uniform in [0,world], per-axis extents U(ext). Draw order per box:
    cx, cy, cz, ex, ey, ez. Computed in float64 and rounded once to float32."""
    r = Rng(seed, STREAM_SCENE)
    u = r.uniform(6 * n).reshape(n, 6)
    c = u[:, :3] * np.asarray(world, dtype=np.float64)
    e = ext[0] + (ext[1] - ext[0]) * u[:, 3:]
    return np.concatenate([c - e / 2, c + e / 2], axis=1).astype(np.float32)


@dataclasses.dataclass(frozen=True)
class CityParams:
    blocks: int = 40
    pitch: float = 10.0
    street: float = 3.0
    n_buildings: int = 2000
    mu: float = 2.0
    sigma: float = 0.6
    foot_lo: float = 2.0
    foot_hi: float = 7.0
    ground_thickness: float = 0.1


def city_boxes(seed: int = 0, p: CityParams = CityParams()) -> np.ndarray:
    """Procedural city: a ground slab plus p.n_buildings boxes on a blocks x blocks lot grid.
    Per building draws (in order): block x, block z, footprint w, footprint d, position x,
    position z, height normal. Heights are lognormal(mu, sigma)."""
    r = Rng(seed, STREAM_SCENE)
    L = p.blocks * p.pitch
    boxes = [np.array([0.0, -p.ground_thickness, 0.0, L, 0.0, L])]
    n = p.n_buildings
    u = r.uniform(6 * n).reshape(n, 6)
    z = r.normal(n)
    lot_w = p.pitch - p.street
    bx = np.floor(u[:, 0] * p.blocks)
    bz = np.floor(u[:, 1] * p.blocks)
    fw = np.minimum(p.foot_lo + (p.foot_hi - p.foot_lo) * u[:, 2], lot_w)
    fd = np.minimum(p.foot_lo + (p.foot_hi - p.foot_lo) * u[:, 3], lot_w)
    x0 = bx * p.pitch + p.street / 2 + u[:, 4] * (lot_w - fw)
    z0 = bz * p.pitch + p.street / 2 + u[:, 5] * (lot_w - fd)
    h = np.exp(p.mu + p.sigma * z)
    b = np.stack([x0, np.zeros(n), z0, x0 + fw, h, z0 + fd], axis=1)
    return np.concatenate([np.stack(boxes), b], axis=0).astype(np.float32)


# ----------------------------------------------------------------------------------------------
# Viewcells
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Viewcell:
    """A cube viewcell of half-size `half` around `centre`, looking along yaw (radians, about +y;
    yaw 0 looks along +z), pitch 0. fov_deg is the camera FOV theta, rot_deg the rotation
    allowance beta (Sec. 3.2, Sec. 4.3)."""
    centre: Tuple[float, float, float]
    half: float
    yaw: float
    fov_deg: float = 60.0
    rot_deg: float = 15.0
    near: float = 0.1
    far: float = 100.0


def city_viewcells(seed: int, count: int, p: CityParams = CityParams(), half: float = 0.5,
                   height=(2.0, 2.0)) -> List[Viewcell]:
    """Viewcells at uniformly random street points. Draws per viewcell (in order): street axis,
    street index, position along, position across, height, yaw."""
    r = Rng(seed, STREAM_VIEWCELL)
    out = []
    L = p.blocks * p.pitch
    for _ in range(count):
        u = r.uniform(6)
        k = 1 + int(math.floor(u[1] * (p.blocks - 1)))
        along = p.pitch + u[2] * (L - 2 * p.pitch)
        across = k * p.pitch + (u[3] - 0.5) * p.street * 0.6
        y = height[0] + u[4] * (height[1] - height[0])
        if u[0] < 0.5:
            c = (across, y, along)
        else:
            c = (along, y, across)
        out.append(Viewcell(centre=c, half=half, yaw=float(u[5] * 2.0 * math.pi)))
    return out


def gt_candidate_offsets(seed: int, vc: Viewcell, n: int) -> np.ndarray:
    """n candidate viewpoints uniform in the viewcell, as offsets (a, b, e) in [-half, half]^3
    along the camera's right, up and forward axes (float64 [n][3]). The viewcell cube is aligned
    with the camera. A consumer that rejects some takes the first M accepted ones, so the sample
    for a smaller M is a prefix of the sample for a larger M."""
    r = Rng(seed, STREAM_GT_POINTS)
    u = r.uniform(3 * n).reshape(n, 3)
    return (2.0 * u - 1.0) * vc.half


# ----------------------------------------------------------------------------------------------
# Networks: layer shape lists (pure data) and initial weights
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Layer:
    name: str
    kind: str        # "subm3" (27 taps), "down2" (8 taps, stride 2), "up2" (8 taps, inverse), "head1" (1 tap),
                     # "down3" (27 taps, stride 2, padding 1), "up3" (27 taps, its inverse)
    cin: int
    cout: int
    relu: bool

    @property
    def taps(self) -> int:
        return {"subm3": 27, "down2": 8, "up2": 8, "head1": 1, "down3": 27, "up3": 27}[self.kind]


def plain_layers(channels: Sequence[int]) -> List[Layer]:
    """A stack of submanifold 3x3x3 layers; ReLU after all but the last."""
    n = len(channels) - 1
    return [Layer(f"conv{i}", "subm3", channels[i], channels[i + 1], i < n - 1) for i in range(n)]


def unet_layers(cin: int, levels: Sequence[int], cout: int, k3: bool = False) -> List[Layer]:
    """Sparse U-Net layer list in canonical order: stem, per level two SubM3 (+ down), then per
    decoder level an inverse conv and two SubM3, then a 1x1 head. k3: the down convs are k = 3,
    stride 2, padding 1 (onto the dilated output set) and the up convs their transposes."""
    dk, uk = ("down3", "up3") if k3 else ("down2", "up2")
    L: List[Layer] = [Layer("stem", "subm3", cin, levels[0], True)]
    nl = len(levels)
    for i in range(nl):
        L.append(Layer(f"enc{i}a", "subm3", levels[i], levels[i], True))
        L.append(Layer(f"enc{i}b", "subm3", levels[i], levels[i], True))
        if i + 1 < nl:
            L.append(Layer(f"down{i}", dk, levels[i], levels[i + 1], True))
    for i in range(nl - 2, -1, -1):
        L.append(Layer(f"up{i}", uk, levels[i + 1], levels[i], True))
        L.append(Layer(f"dec{i}a", "subm3", levels[i], levels[i], True))
        L.append(Layer(f"dec{i}b", "subm3", levels[i], levels[i], True))
    L.append(Layer("head", "head1", levels[0], cout, False))
    return L


def kaiming_uniform(layers: Sequence[Layer], seed: int = 0, bias_scale: float = 0.0):
    """Per layer, weights [taps][cin][cout] ~ U(-b, b) with b = sqrt(6 / (cin * taps)), drawn in
    layer order and row-major order from one stream, rounded once to float32. Biases are zero
    unless bias_scale > 0 (then U(-bias_scale, bias_scale) from a second stream)."""
    r = Rng(seed, STREAM_WEIGHTS)
    rb = Rng(seed, STREAM_MISC)
    ws, bs = [], []
    for l in layers:
        n = l.taps * l.cin * l.cout
        bound = math.sqrt(6.0 / (l.cin * l.taps))
        w = (2.0 * r.uniform(n) - 1.0) * bound
        ws.append(w.reshape(l.taps, l.cin, l.cout).astype(np.float32))
        if bias_scale > 0:
            bs.append(((2.0 * rb.uniform(l.cout) - 1.0) * bias_scale).astype(np.float32))
        else:
            bs.append(np.zeros(l.cout, dtype=np.float32))
    return ws, bs


# ----------------------------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    W: int
    H: int
    D: int
    d: int
    in_ch: int
    supersample: int
    layers: Tuple[Layer, ...]

    @property
    def feat_ch(self) -> int:
        return self.in_ch * self.d ** 3


def workload(name: str) -> Workload:
    if name == "plain64":      # 64x64x32 froxels, d=2, occupancy only, 4 SubM3 layers
        return Workload(name, 64, 64, 32, 2, 1, 8, tuple(plain_layers([8, 16, 32, 16, 8])))
    if name == "city256":      # 256x256x128 froxels, d=4, occupancy + depth, U-Net 32/64/128/256
        return Workload(name, 256, 256, 128, 4, 2, 8, tuple(unet_layers(128, [32, 64, 128, 256], 64)))
    if name == "city256_k3":   # city256 with k = 3, stride 2 down convs (dilated levels) and their transposes
        return Workload(name, 256, 256, 128, 4, 2, 8, tuple(unet_layers(128, [32, 64, 128, 256], 64, k3=True)))
    if name == "city512":      # 512x512x192 froxels, d=8, occupancy + depth, U-Net 64/128/256/512
        return Workload(name, 512, 512, 192, 8, 2, 4, tuple(unet_layers(1024, [64, 128, 256, 512], 512)))
    if name == "paper256":     # the paper's grid: 256^3 froxels, d=16 (4096 ch), stem to ~200 ch, 2 levels
        return Workload(name, 256, 256, 256, 16, 1, 8, tuple(unet_layers(4096, [192, 256], 4096)))
    if name == "paper64":      # the same network at d=16 on a 64^3 grid (4^3 coarse sites)
        return Workload(name, 64, 64, 64, 16, 1, 8, tuple(unet_layers(4096, [192, 256], 4096)))
    if name == "paper256_d8":  # the paper's grid at d=8 (512 ch), the same U-Net
        return Workload(name, 256, 256, 256, 8, 1, 8, tuple(unet_layers(512, [192, 256], 512)))
    if name == "paper64_d8":   # the same network on a 64^3 grid (8^3 coarse sites)
        return Workload(name, 64, 64, 64, 8, 1, 8, tuple(unet_layers(512, [192, 256], 512)))
    if name == "paper256_d32":  # the paper's grid at d=32 (32,768 ch), the same U-Net
        return Workload(name, 256, 256, 256, 32, 1, 8, tuple(unet_layers(32768, [192, 256], 32768)))
    if name == "paper64_d32":  # the same network on a 64^3 grid (2^3 coarse sites)
        return Workload(name, 64, 64, 64, 32, 1, 8, tuple(unet_layers(32768, [192, 256], 32768)))
    if name == "paper256_d1":  # the paper256 network without interleave: one channel per froxel
        return Workload(name, 256, 256, 256, 1, 1, 8, tuple(unet_layers(1, [192, 256], 1)))
    if name == "nointerleave64":  # d=1 on a 64^3 grid, narrow widths (small enough for the oracle)
        return Workload(name, 64, 64, 64, 1, 1, 8, tuple(unet_layers(1, [16, 32], 1)))
    raise KeyError(name)


def plain64_scene():
    """40 boxes in a 100x20x100 world (seed 0) and the viewcell at (55,10,15) looking along +z,
    1x1x1 world units (half-size 0.5)."""
    return random_boxes(0, 40), Viewcell(centre=(55.0, 10.0, 15.0), half=0.5, yaw=0.0)


CITY_LARGE = CityParams(n_buildings=10000, mu=2.3, sigma=0.7)
