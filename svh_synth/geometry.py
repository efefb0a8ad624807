"""Seeded voxel geometries shaped like the paper's test structures (Sec. III).

Array layout everywhere: ``occ[z, y, x]`` (C order, x fastest), matching the
library's row-major, x-fastest grid convention. A voxel's linear index is
``x + Kx * (y + Ky * z)``.

A port terminal is a list of voxel faces, each encoded as
``voxel_linear_index * 6 + face`` with face order -x, +x, -y, +y, -z, +z.
A port drives a unit potential difference between its ``plus`` faces and its
``minus`` faces; the other ports are shorted (Y-parameter convention).

Only geometry and material values are produced here: the face-node numbering,
incidence matrix and all arithmetic of the method live in the code under test
and, independently, in the oracle.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

MU0 = 4e-7 * np.pi  # permeability of free space (H/m); mu = mu0 in the paper (Sec. II.A)

FACE_MX, FACE_PX, FACE_MY, FACE_PY, FACE_MZ, FACE_PZ = range(6)


@dataclass
class Port:
    plus: np.ndarray   # int32 face codes
    minus: np.ndarray  # int32 face codes


@dataclass
class Structure:
    name: str
    Kx: int
    Ky: int
    Kz: int
    dx: float                     # voxel edge (m)
    occ: np.ndarray               # uint8 [Kz, Ky, Kx]
    lam: np.ndarray               # float64 London depth (m) [Kz, Ky, Kx]
    sigma0: np.ndarray            # float64 normal conductivity (S/m) [Kz, Ky, Kx]
    ports: List[Port] = field(default_factory=list)
    freqs: Tuple[float, ...] = (1e9,)

    @property
    def Kt(self) -> int:
        return self.Kx * self.Ky * self.Kz

    @property
    def K(self) -> int:
        return int(self.occ.sum())


def _lin(Kx, Ky, x, y, z):
    return x + Kx * (y + Ky * z)


def box_faces(Kx, Ky, x0, x1, y0, y1, z0, z1, face) -> np.ndarray:
    """Face codes of one side of the voxel box [x0,x1]x[y0,y1]x[z0,z1] (inclusive).

    The side is given by ``face``; e.g. FACE_PX lists the +x faces of the
    voxels in the box's x = x1 slice."""
    xs = np.arange(x0, x1 + 1)
    ys = np.arange(y0, y1 + 1)
    zs = np.arange(z0, z1 + 1)
    if face == FACE_MX:
        xs = np.array([x0])
    elif face == FACE_PX:
        xs = np.array([x1])
    elif face == FACE_MY:
        ys = np.array([y0])
    elif face == FACE_PY:
        ys = np.array([y1])
    elif face == FACE_MZ:
        zs = np.array([z0])
    elif face == FACE_PZ:
        zs = np.array([z1])
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return (_lin(Kx, Ky, X, Y, Z).ravel() * 6 + face).astype(np.int32)


def _empty(name, Kx, Ky, Kz, dx, freqs):
    occ = np.zeros((Kz, Ky, Kx), np.uint8)
    lam = np.zeros((Kz, Ky, Kx), np.float64)
    sig = np.zeros((Kz, Ky, Kx), np.float64)
    return Structure(name, Kx, Ky, Kz, dx, occ, lam, sig, [], tuple(freqs))


def _fill(s: Structure, x0, x1, y0, y1, z0, z1, lam, sigma0):
    s.occ[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1] = 1
    s.lam[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1] = lam
    s.sigma0[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1] = sigma0


def bar(Kx, Ky, Kz, x0, x1, y0, y1, z0, z1, dx=0.1e-6, lam=90e-9,
        sigma0=1e7, freqs=(1e9,), name="bar") -> Structure:
    """Straight bar along x, one port from its -x end face (minus) to its +x end face (plus)."""
    s = _empty(name, Kx, Ky, Kz, dx, freqs)
    _fill(s, x0, x1, y0, y1, z0, z1, lam, sigma0)
    s.ports.append(Port(plus=box_faces(Kx, Ky, x0, x1, y0, y1, z0, z1, FACE_PX),
                        minus=box_faces(Kx, Ky, x0, x1, y0, y1, z0, z1, FACE_MX)))
    return s


def strip_cfg1() -> Structure:
    """16x16x4 grid, 0.1 um voxels, strip 16x4x2 at x 0-15, y 6-9, z 1-2.

    lambda = 90 nm, sigma_n = 1e7 S/m, f = 1 GHz; one port between the x = 0
    end face (minus) and the x = 16 end face (plus)."""
    return bar(16, 16, 4, 0, 15, 6, 9, 1, 2, dx=0.1e-6, lam=90e-9, sigma0=1e7,
               freqs=(1e9,), name="strip16x16x4")


def random_blob(seed, Kx, Ky, Kz, fill=0.5, dx=0.1e-6, lam_range=(50e-9, 150e-9),
                sigma0=1e7) -> Structure:
    """Random occupancy (for operator parity tests; no ports) with per-voxel lambda."""
    rng = np.random.default_rng(seed)
    s = _empty(f"blob{seed}", Kx, Ky, Kz, dx, (1e9,))
    s.occ[...] = (rng.random((Kz, Ky, Kx)) < fill).astype(np.uint8)
    s.lam[...] = rng.uniform(*lam_range, size=(Kz, Ky, Kx)) * s.occ
    s.sigma0[...] = sigma0 * s.occ
    return s


def _meander_cells(x0, y0, n_legs, leg_len, width=4, pitch=8):
    """Voxel rectangles (x0,x1,y0,y1) of a meander whose legs run along y.

    Returns (rects, start_patch, end_patch, end_at_top); the patches are the
    width x width squares at the two free ends."""
    rects = []
    y1 = y0 + leg_len - 1
    for i in range(n_legs):
        xa = x0 + pitch * i
        rects.append((xa, xa + width - 1, y0, y1))
        if i < n_legs - 1:
            if i % 2 == 0:
                rects.append((xa, xa + pitch + width - 1, y1 - width + 1, y1))
            else:
                rects.append((xa, xa + pitch + width - 1, y0, y0 + width - 1))
    start = (x0, x0 + width - 1, y0, y0 + width - 1)
    xl = x0 + pitch * (n_legs - 1)
    end_at_top = (n_legs - 2) % 2 == 1 if n_legs >= 2 else True
    if end_at_top:
        end = (xl, xl + width - 1, y1 - width + 1, y1)
    else:
        end = (xl, xl + width - 1, y0, y0 + width - 1)
    return rects, start, end, end_at_top


def meander_cfg2(seed=202, Kx=256, Ky=256, Kz=8, dx=0.1e-6) -> Structure:
    """Thin-film meander over a ground plane with holes (cfg 2 shape).

    Ground z 0-1 with seeded square holes (side 4-16, about 15 % open area),
    gap z 2-3, meander z 4-5 (width 4, pitch 8, 8-20 turns, seeded leg
    length, at least 16 voxels from the border); a via joins one meander end
    to ground; one port sits between the other meander end (its bottom faces)
    and the ground top faces right below it. lambda per layer ~ U[50,150] nm."""
    rng = np.random.default_rng(seed)
    s = _empty(f"meander{Kx}x{Ky}x{Kz}_s{seed}", Kx, Ky, Kz, dx, (1e9,))
    lam_g, lam_m, lam_v = rng.uniform(50e-9, 150e-9, size=3)
    n_turns = int(rng.integers(8, 21))
    n_legs = n_turns + 1
    width_x = 8 * (n_legs - 1) + 4
    x0 = int(rng.integers(16, Kx - 16 - width_x + 1))
    leg_len = int(rng.integers(64, Ky - 32 + 1))
    y0 = int(rng.integers(16, Ky - 16 - leg_len + 1))
    rects, start, end, _ = _meander_cells(x0, y0, n_legs, leg_len)
    # ground plane
    _fill(s, 0, Kx - 1, 0, Ky - 1, 0, 1, lam_g, 1e7)
    keep = [start, end]
    open_target = 0.15 * Kx * Ky
    opened = 0
    tries = 0
    while opened < open_target and tries < 10000:
        tries += 1
        a = int(rng.integers(4, 17))
        hx = int(rng.integers(0, Kx - a + 1))
        hy = int(rng.integers(0, Ky - a + 1))
        bad = any(hx <= kx1 + 4 and hx + a - 1 >= kx0 - 4 and hy <= ky1 + 4 and hy + a - 1 >= ky0 - 4
                  for (kx0, kx1, ky0, ky1) in keep)
        if bad:
            continue
        before = int(s.occ[0, hy:hy + a, hx:hx + a].sum())
        s.occ[0:2, hy:hy + a, hx:hx + a] = 0
        opened += before
    s.lam[0:2] *= s.occ[0:2]
    s.sigma0[0:2] *= s.occ[0:2]
    for (a0, a1, b0, b1) in rects:
        _fill(s, a0, a1, b0, b1, 4, 5, lam_m, 1e7)
    # via at the end patch down to ground
    ex0, ex1, ey0, ey1 = end
    _fill(s, ex0, ex1, ey0, ey1, 2, 3, lam_v, 1e7)
    sx0, sx1, sy0, sy1 = start
    plus = box_faces(Kx, Ky, sx0, sx1, sy0, sy1, 4, 5, FACE_MZ)
    minus = box_faces(Kx, Ky, sx0, sx1, sy0, sy1, 0, 1, FACE_PZ)
    s.ports.append(Port(plus=plus, minus=minus))
    return s


def pair_cfg4(seed=404, Kx=128, Ky=128, Kz=16, dx=0.1e-6) -> Structure:
    """Two meander inductors at z 2-3 and z 8-9 with overlapping footprints.

    Per-voxel lambda is log-normal (median 90 nm, sigma_ln = 0.3). Each
    meander carries one port between its two free end faces (minus at the
    start, plus at the end)."""
    rng = np.random.default_rng(seed)
    s = _empty(f"pair{Kx}x{Ky}x{Kz}_s{seed}", Kx, Ky, Kz, dx, (1e9,))
    for zl in (2, 8):
        n_legs = int(rng.integers(5, 10))
        width_x = 8 * (n_legs - 1) + 4
        x0 = int(rng.integers(8, Kx - 8 - width_x + 1))
        leg_len = int(rng.integers(40, Ky - 16 + 1))
        y0 = int(rng.integers(8, Ky - 8 - leg_len + 1))
        rects, start, end, end_at_top = _meander_cells(x0, y0, n_legs, leg_len)
        for (a0, a1, b0, b1) in rects:
            _fill(s, a0, a1, b0, b1, zl, zl + 1, 90e-9, 1e7)
        sx0, sx1, sy0, sy1 = start
        ex0, ex1, ey0, ey1 = end
        minus = box_faces(Kx, Ky, sx0, sx1, sy0, sy0, zl, zl + 1, FACE_MY)
        if end_at_top:
            plus = box_faces(Kx, Ky, ex0, ex1, ey1, ey1, zl, zl + 1, FACE_PY)
        else:
            plus = box_faces(Kx, Ky, ex0, ex1, ey0, ey0, zl, zl + 1, FACE_MY)
        s.ports.append(Port(plus=plus, minus=minus))
    ln = rng.normal(np.log(90e-9), 0.3, size=s.occ.shape)
    s.lam[...] = np.exp(ln) * s.occ
    return s


def _bend(s, rng, cx, cy, z0, sec, arm_x, arm_y, lam, sigma0):
    """L-bend: arm along +x from the corner square, arm along +y from it."""
    Kx, Ky = s.Kx, s.Ky
    _fill(s, cx, cx + arm_x - 1, cy, cy + sec - 1, z0, z0 + sec - 1, lam, sigma0)
    _fill(s, cx, cx + sec - 1, cy, cy + arm_y - 1, z0, z0 + sec - 1, lam, sigma0)
    minus = box_faces(Kx, Ky, cx + arm_x - 1, cx + arm_x - 1, cy, cy + sec - 1, z0, z0 + sec - 1, FACE_PX)
    plus = box_faces(Kx, Ky, cx, cx + sec - 1, cy + arm_y - 1, cy + arm_y - 1, z0, z0 + sec - 1, FACE_PY)
    return Port(plus=plus, minus=minus)


def batch_cfg3(seed=303, n_items=64) -> List[Structure]:
    """Unevenly sized items: Kx, Ky ~ U{32..128}, Kz ~ U{8..16}.

    Half are nested sharp L-bends (square section 4-8 voxels, shaped like the
    paper's 90-degree bend), half are parallel meander traces; 4-8 ports per
    item (one per bend or trace); frequencies 1, 10 and 50 GHz."""
    rng = np.random.default_rng(seed)
    items = []
    for it in range(n_items):
        Kx = int(rng.integers(32, 129))
        Ky = int(rng.integers(32, 129))
        Kz = int(rng.integers(8, 17))
        s = _empty(f"item{it}_{Kx}x{Ky}x{Kz}", Kx, Ky, Kz, 0.1e-6, (1e9, 10e9, 50e9))
        p = int(rng.integers(4, 9))
        lam = float(rng.uniform(50e-9, 150e-9))
        if it % 2 == 0:
            sec = int(rng.integers(4, 9))
            avail = min(Kx, Ky) - 4
            sec = min(sec, Kz - 2)
            while p * (sec + 2) > avail:
                if sec > 1:
                    sec -= 1
                else:
                    p -= 1
            z0 = (Kz - sec) // 2
            for j in range(p):
                # nested bends: bend j has its corner at (c, c); its arms run to
                # the far +x and +y borders, parallel to and clear of bend j-1
                c = 2 + j * (sec + 2)
                s.ports.append(_bend(s, rng, c, c, z0, sec, Kx - 2 - c, Ky - 2 - c, lam, 1e7))
        else:
            band = (Ky - 4) // p
            w = max(1, min(2, band // 4))
            z0 = (Kz - 2) // 2
            for j in range(p):
                yb = 2 + j * band
                h = band - 2
                # zig-zag trace in its own band: legs along y of height h, pitch 2w+1... along x
                pitch = 2 * w + 1
                n_legs = max(2, (Kx - 4) // pitch)
                x = 2
                for i in range(n_legs):
                    xa = x + pitch * i
                    _fill(s, xa, xa + w - 1, yb, yb + h - 1, z0, z0 + 1, lam, 1e7)
                    if i < n_legs - 1:
                        if i % 2 == 0:
                            _fill(s, xa, xa + pitch + w - 1, yb + h - w, yb + h - 1, z0, z0 + 1, lam, 1e7)
                        else:
                            _fill(s, xa, xa + pitch + w - 1, yb, yb + w - 1, z0, z0 + 1, lam, 1e7)
                minus = box_faces(Kx, Ky, x, x + w - 1, yb, yb, z0, z0 + 1, FACE_MY)
                xl = x + pitch * (n_legs - 1)
                if (n_legs - 2) % 2 == 1:
                    plus = box_faces(Kx, Ky, xl, xl + w - 1, yb + h - 1, yb + h - 1, z0, z0 + 1, FACE_PY)
                else:
                    plus = box_faces(Kx, Ky, xl, xl + w - 1, yb, yb, z0, z0 + 1, FACE_MY)
                s.ports.append(Port(plus=plus, minus=minus))
        items.append(s)
    return items


def esfq_cfg5(seed=505, Kx=512, Ky=512, Kz=24, dx=0.5e-6, n_ports=16) -> Structure:
    """eSFQ-like multilayer block (cfg 5 shape), 0.5 um voxels.

    Ground z 0-1 perforated by a 25 % hole grid (8x8 holes, period 16);
    wiring layers at z 6-7, 12-13 and 18-19 with seeded Manhattan wires of
    width 2-6. Each wire drops to ground through a via at its start; its
    port sits between the bottom faces of its far end and the ground top
    faces right below. lambda = 90 nm everywhere."""
    rng = np.random.default_rng(seed)
    s = _empty(f"esfq{Kx}x{Ky}x{Kz}_s{seed}", Kx, Ky, Kz, dx, (1e9,))
    layers = [6, 12, 18]
    taken = np.zeros((Kz, Ky, Kx), bool)
    keep_solid = []
    placed = 0
    tries = 0
    while placed < n_ports and tries < 5000:
        tries += 1
        zl = layers[int(rng.integers(0, 3))]
        w = int(rng.integers(2, 7))
        nseg = int(rng.integers(2, 6))
        x = int(rng.integers(24, Kx - 24 - w))
        y = int(rng.integers(24, Ky - 24 - w))
        rects = []
        horiz = bool(rng.integers(0, 2))
        start = (x, x + w - 1, y, y + w - 1)
        ok = True
        for _ in range(nseg):
            L = int(rng.integers(20, 120))
            sgn = 1 if rng.integers(0, 2) else -1
            if horiz:
                nx = int(np.clip(x + sgn * L, 24, Kx - 24 - w))
                rects.append((min(x, nx), max(x, nx) + w - 1, y, y + w - 1))
                x = nx
            else:
                ny = int(np.clip(y + sgn * L, 24, Ky - 24 - w))
                rects.append((x, x + w - 1, min(y, ny), max(y, ny) + w - 1))
                y = ny
            horiz = not horiz
        end = (x, x + w - 1, y, y + w - 1)
        if abs(end[0] - start[0]) < 8 and abs(end[2] - start[2]) < 8:
            continue
        trial = np.zeros_like(taken)
        for (a0, a1, b0, b1) in rects:
            trial[zl:zl + 2, b0:b1 + 1, a0:a1 + 1] = True
        sx0, sx1, sy0, sy1 = start
        trial[2:zl, sy0:sy1 + 1, sx0:sx1 + 1] = True
        # clearance of 2 voxels to everything placed before
        grown = trial.copy()
        for ax in (1, 2):
            for sh in (-2, -1, 1, 2):
                grown |= np.roll(trial, sh, axis=ax)
        grown[max(zl - 1, 2):zl + 3] |= grown[zl:zl + 1].any(axis=0)
        if (grown & taken).any():
            ok = False
        if not ok:
            continue
        taken |= trial
        for (a0, a1, b0, b1) in rects:
            _fill(s, a0, a1, b0, b1, zl, zl + 1, 90e-9, 1e7)
        _fill(s, sx0, sx1, sy0, sy1, 2, zl - 1, 90e-9, 1e7)
        ex0, ex1, ey0, ey1 = end
        keep_solid += [start, end]
        plus = box_faces(Kx, Ky, ex0, ex1, ey0, ey1, zl, zl + 1, FACE_MZ)
        minus = box_faces(Kx, Ky, ex0, ex1, ey0, ey1, 0, 1, FACE_PZ)
        s.ports.append(Port(plus=plus, minus=minus))
        placed += 1
    # perforated ground: 8x8 holes with period 16 (25 % open), solid under vias and ports
    g = np.ones((Ky, Kx), bool)
    for hy in range(4, Ky - 8, 16):
        for hx in range(4, Kx - 8, 16):
            g[hy:hy + 8, hx:hx + 8] = False
    for (a0, a1, b0, b1) in keep_solid:
        g[max(b0 - 4, 0):b1 + 5, max(a0 - 4, 0):a1 + 5] = True
    s.occ[0:2] = g[None].astype(np.uint8)
    s.lam[0:2] = 90e-9 * g[None]
    s.sigma0[0:2] = 1e7 * g[None]
    return s
