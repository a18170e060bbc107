"""Seeded synthetic periodic lattice cells (binary voxel fields).

These are the inputs of the homogenization problem: a periodic N^3 cell of solid (1) and
void (0) voxels, stored as a uint8 array indexed [z, y, x] (x fastest in memory).
The module holds no part of the solver's arithmetic; it is imported by the tests, the
benchmark and the oracle checks alike so that both sides see the same voxels.

Families follow the paper's data description (Sec. 5, "Datasets"; App. C: TPMS, plate
(sheet) lattices and strut/truss lattices, volume fractions 10-30 %), plus spinodal cells
from a Gaussian random field. The paper's datasets are not available; these generators
stand in for them with the same shapes and volume-fraction ranges.

Rules used everywhere:
  * voxel centres are at X = 2*pi*(i + 1/2)/N for level-set families and at (i + 1/2)/N
    for strut families;
  * a level set is thresholded so that exactly round(phi * N^3) voxels are solid: the
    voxels with the smallest field value win, ties broken by linear index (stable sort);
  * optionally only the largest face-connected (6-connected, periodic) solid component is
    kept, so that the stiffness has no floating islands.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

__all__ = [
    "gyroid_field", "schwarz_p_field", "diamond_field", "tpms_network", "tpms_plate",
    "truss", "spinodal", "largest_component", "laminate_z", "rods_x", "random_binary",
    "batch_cell", "unet_init",
    "mixed_cell", "FAMILIES",
]


def _grid(n: int):
    c = 2.0 * np.pi * (np.arange(n, dtype=np.float64) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return x, y, z


def gyroid_field(n: int) -> np.ndarray:
    x, y, z = _grid(n)
    return np.sin(x) * np.cos(y) + np.sin(y) * np.cos(z) + np.sin(z) * np.cos(x)


def schwarz_p_field(n: int) -> np.ndarray:
    x, y, z = _grid(n)
    return np.cos(x) + np.cos(y) + np.cos(z)


def diamond_field(n: int) -> np.ndarray:
    x, y, z = _grid(n)
    return (np.sin(x) * np.sin(y) * np.sin(z) + np.sin(x) * np.cos(y) * np.cos(z)
            + np.cos(x) * np.sin(y) * np.cos(z) + np.cos(x) * np.cos(y) * np.sin(z))


_TPMS = {"gyroid": gyroid_field, "schwarz_p": schwarz_p_field, "diamond": diamond_field}


def _lowest(values: np.ndarray, phi: float) -> np.ndarray:
    """Solid = the round(phi*N^3) voxels with the smallest value (stable by linear index):
    everything below the count-th smallest value, then the earliest ties at that value."""
    flat = values.reshape(-1)
    count = int(round(phi * flat.size))
    out = np.zeros(flat.size, dtype=np.uint8)
    if count <= 0:
        return out.reshape(values.shape)
    if count >= flat.size:
        out[:] = 1
        return out.reshape(values.shape)
    kth = np.partition(flat, count - 1)[count - 1]
    below = flat < kth
    out[below] = 1
    ties = np.flatnonzero(flat == kth)
    out[ties[: count - int(below.sum())]] = 1
    return out.reshape(values.shape)


def tpms_network(family: str, n: int, phi: float) -> np.ndarray:
    """Network TPMS: solid where f < t, t chosen for volume fraction phi."""
    return _lowest(_TPMS[family](n), phi)


def tpms_plate(family: str, n: int, phi: float) -> np.ndarray:
    """Plate (sheet) TPMS: solid where |f| < w, w chosen for volume fraction phi."""
    return _lowest(np.abs(_TPMS[family](n)), phi)


def _segments(kind: str) -> np.ndarray:
    if kind == "bcc":
        a = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
        b = np.array([[1, 1, 1], [0, 1, 1], [1, 0, 1], [1, 1, 0]], dtype=np.float64)
        return np.stack([a, b], axis=1)
    if kind == "octet":
        # FCC sites of the unit cell (corners and face centres, periodic); struts join
        # every pair of sites at the nearest-neighbour distance sqrt(2)/2.
        base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
        shifts = np.array([[i, j, k] for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)],
                          dtype=np.float64)
        sites = (base[None, :, :] + shifts[:, None, :]).reshape(-1, 3)
        segs = []
        for i, p in enumerate(base):
            d = np.linalg.norm(sites - p, axis=1)
            for q in sites[np.abs(d - np.sqrt(0.5)) < 1e-9]:
                key = tuple(np.round(np.sort(np.stack([p, q]), axis=0).ravel(), 6))
                segs.append((key, (p, q)))
        uniq = {}
        for key, seg in segs:
            mid = tuple(np.round(((seg[0] + seg[1]) / 2.0) % 1.0, 6))
            uniq.setdefault(mid, seg)
        return np.array([[s[0], s[1]] for s in uniq.values()], dtype=np.float64)
    raise ValueError(kind)


def truss(kind: str, n: int, radius: float) -> np.ndarray:
    """Strut lattice: solid where the periodic distance from the voxel centre to any strut
    axis is at most `radius` (in units of the cell size). Each periodic image of a strut is
    only evaluated on the voxels inside its bounding box grown by the radius (the only
    voxels it can reach)."""
    c = (np.arange(n, dtype=np.float64) + 0.5) / n
    best = np.full((n, n, n), np.inf)
    for a, b in _segments(kind):
        ab = b - a
        l2 = float(ab @ ab)
        for sx in (-1, 0, 1):
            for sy in (-1, 0, 1):
                for sz in (-1, 0, 1):
                    s = np.array([sx, sy, sz], dtype=np.float64)
                    lo = np.minimum(a, b) + s - radius
                    hi = np.maximum(a, b) + s + radius
                    i0 = np.maximum(np.ceil(lo * n - 0.5), 0).astype(int)
                    i1 = np.minimum(np.floor(hi * n - 0.5), n - 1).astype(int)
                    if (i1 < i0).any():
                        continue
                    zc, yc, xc = (c[i0[2]:i1[2] + 1], c[i0[1]:i1[1] + 1], c[i0[0]:i1[0] + 1])
                    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
                    q = np.stack([X, Y, Z], axis=-1) - (a + s)
                    t = np.clip(q @ ab / l2, 0.0, 1.0)
                    d = q - t[..., None] * ab
                    d2 = np.einsum("...i,...i->...", d, d)
                    sub = best[i0[2]:i1[2] + 1, i0[1]:i1[1] + 1, i0[0]:i1[0] + 1]
                    np.minimum(sub, d2, out=sub)
    return (best <= radius * radius).astype(np.uint8)


def spinodal(n: int, phi: float, wavenumber: int, rng: np.random.Generator,
             modes: int = 64) -> np.ndarray:
    """Gaussian-random-field spinodal cell: sum of `modes` cosines with integer wave vectors
    on the shell |k| in [w - 1/2, w + 1/2] and random phases, thresholded at phi.
    The wavenumber is clamped to N/4 so that a wavelength spans at least 4 voxels."""
    w = min(int(wavenumber), n // 4)
    r = int(np.ceil(w + 0.5))
    ks = np.array([[i, j, k] for i in range(-r, r + 1) for j in range(-r, r + 1)
                   for k in range(-r, r + 1)], dtype=np.int64)
    norm = np.linalg.norm(ks, axis=1)
    shell = ks[(norm >= w - 0.5) & (norm <= w + 0.5)]
    pick = shell[rng.integers(0, len(shell), size=modes)]
    theta = rng.uniform(0.0, 2.0 * np.pi, size=modes)
    c = (np.arange(n, dtype=np.float64) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    f = np.zeros((n, n, n))
    for kv, th in zip(pick, theta):
        f += np.cos(2.0 * np.pi * (kv[0] * x + kv[1] * y + kv[2] * z) + th)
    return _lowest(f, phi)


def largest_component(vox: np.ndarray) -> np.ndarray:
    """Keep only the largest face-connected solid component, with periodic wrap."""
    lab, count = ndimage.label(vox.astype(bool))
    if count <= 1:
        return vox.astype(np.uint8)
    parent = np.arange(count + 1)

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    for axis in range(3):
        a = np.take(lab, 0, axis=axis).ravel()
        b = np.take(lab, -1, axis=axis).ravel()
        for u, v in zip(a[(a > 0) & (b > 0)], b[(a > 0) & (b > 0)]):
            ru, rv = find(int(u)), find(int(v))
            if ru != rv:
                parent[max(ru, rv)] = min(ru, rv)
    roots = np.array([find(i) for i in range(count + 1)])
    merged = roots[lab]
    sizes = np.bincount(merged.ravel(), minlength=count + 1)
    sizes[0] = 0
    keep = int(np.argmax(sizes))
    return (merged == keep).astype(np.uint8)


def laminate_z(n: int, solid_layers) -> np.ndarray:
    """Plates normal to z: every voxel whose z index is listed is solid."""
    v = np.zeros((n, n, n), dtype=np.uint8)
    v[list(solid_layers), :, :] = 1
    return v


def rods_x(n: int, width: int, count_y: int = 1, count_z: int = 1) -> np.ndarray:
    """Square rods of `width` voxels running along x, on a count_y x count_z array."""
    v = np.zeros((n, n, n), dtype=np.uint8)
    sy, sz = n // count_y, n // count_z
    for j in range(count_y):
        for k in range(count_z):
            v[k * sz:k * sz + width, j * sy:j * sy + width, :] = 1
    return v


def random_binary(n: int, phi: float, rng: np.random.Generator) -> np.ndarray:
    return (rng.random((n, n, n)) < phi).astype(np.uint8)


FAMILIES = ("gyroid", "schwarz_p", "diamond", "plate_gyroid", "plate_schwarz_p",
            "plate_diamond", "bcc", "octet", "spinodal")


def mixed_cell(seed: int, n: int, families=FAMILIES, phi_range=(0.10, 0.40),
               radius_range=(0.04, 0.10), wavenumber_range=(8, 16), keep_largest=True):
    """One cell of the seeded mixed workload. Returns (voxels, description dict)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    fam = families[int(rng.integers(0, len(families)))]
    phi = float(rng.uniform(*phi_range))
    desc = {"family": fam, "n": n, "seed": seed}
    if fam in _TPMS:
        vox = tpms_network(fam, n, phi)
        desc["phi_target"] = phi
    elif fam.startswith("plate_"):
        vox = tpms_plate(fam[len("plate_"):], n, phi)
        desc["phi_target"] = phi
    elif fam in ("bcc", "octet"):
        r = float(rng.uniform(*radius_range))
        vox = truss(fam, n, r)
        desc["radius"] = r
    elif fam == "spinodal":
        w = int(rng.integers(wavenumber_range[0], wavenumber_range[1] + 1))
        vox = spinodal(n, phi, w, rng)
        desc["phi_target"] = phi
        desc["wavenumber"] = min(w, n // 4)
    else:
        raise ValueError(fam)
    if keep_largest:
        vox = largest_component(vox)
    desc["phi"] = float(vox.mean())
    return vox, desc


BATCH_RESOLUTIONS = (32, 48, 64, 96, 128)


def batch_cell(seed: int, resolutions=BATCH_RESOLUTIONS):
    """One cell of the uneven-resolution batch: N drawn uniformly from `resolutions` by its
    own PCG64(seed) stream, then mixed_cell(seed, N) over all families (spinodal included)."""
    rng = np.random.default_rng(np.random.PCG64([seed, 1]))
    n = int(resolutions[int(rng.integers(0, len(resolutions)))])
    return mixed_cell(seed, n, families=FAMILIES)


def unet_init(rows, seed: int) -> np.ndarray:
    """Seeded initial parameters of the initializer network (float32, flat): for each layer
    row (..., cin, cout) the weights W [27][cin][cout] drawn N(0, 2 / (27 cin)) (He
    initialisation) by a PCG64(seed) stream, then the biases b [cout] = 0."""
    rng = np.random.default_rng(np.random.PCG64([seed, 7]))
    parts = []
    for r in rows:
        cin, cout = int(r[4]), int(r[5])
        parts.append(rng.normal(0.0, np.sqrt(2.0 / (27 * cin)), size=27 * cin * cout))
        parts.append(np.zeros(cout))
    return np.concatenate(parts).astype(np.float32)
