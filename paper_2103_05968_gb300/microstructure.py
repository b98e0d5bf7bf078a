"""Seeded synthetic microstructures (crack-resistance fields gamma on a voxel grid).

This module only builds inputs. It holds none of the solver's arithmetic and
imports neither the CUDA binding nor the oracle, so both sides of every parity
test draw their inputs from here.

Conventions (Sec. 2.2 of the paper): the grid has N1 x N2 x N3 voxels of unit
edge, the array is C-ordered with shape (N1, N2, N3) indexed [i, j, k] = (x, y, z),
and gamma is sampled at the voxel centres ((i + 1/2), (j + 1/2), (k + 1/2)).
A voxel belongs to a shape iff its centre lies strictly inside the shape, with
periodic wrap-around of the cell.

Random numbers come from ``numpy.random.default_rng(seed)`` (PCG64 seeded through
SeedSequence), so a seed fixes every field bit for bit on any machine.
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "single_sphere",
    "boolean_spheres",
    "short_fibres",
    "lognormal_field",
    "laminate",
    "random_two_phase",
    "uniform_random",
    "disks_2d",
    "relaxed_spheres",
    "porous_spheres",
    "sand_binder",
    "config_single_sphere_32",
    "config_boolean_spheres_128",
    "config_short_fibres_512",
]


def _centres(n):
    return [np.arange(m, dtype=np.float64) + 0.5 for m in n]


def _periodic_delta(x, c, length):
    d = x - c
    d -= length * np.round(d / length)
    return d


def _stamp_ball(mask, centre, radius):
    """Set every voxel whose centre is strictly inside the periodic ball."""
    n = mask.shape
    r = float(radius)
    lo = [int(math.floor(centre[a] - r - 1)) for a in range(3)]
    hi = [int(math.ceil(centre[a] + r + 1)) for a in range(3)]
    idx = [np.arange(lo[a], hi[a] + 1) for a in range(3)]
    d2 = None
    for a in range(3):
        da = (idx[a] + 0.5) - centre[a]
        shape = [1, 1, 1]
        shape[a] = -1
        term = (da * da).reshape(shape)
        d2 = term if d2 is None else d2 + term
    inside = d2 < r * r
    ii, jj, kk = np.nonzero(inside)
    sel = ((idx[0][ii] % n[0]), (idx[1][jj] % n[1]), (idx[2][kk] % n[2]))
    before = int(np.count_nonzero(mask[sel]))
    mask[sel] = True
    return int(np.count_nonzero(mask[sel])) - before


def single_sphere(n, centre, radius, gamma_sphere, gamma_matrix, dtype=np.float64):
    """One ball of the given radius (voxel units) in a homogeneous matrix."""
    n = tuple(int(m) for m in n)
    mask = np.zeros(n, dtype=bool)
    _stamp_ball(mask, np.asarray(centre, dtype=np.float64), radius)
    g = np.where(mask, gamma_sphere, gamma_matrix).astype(dtype)
    return g


def boolean_spheres(n, radius, volume_fraction, gamma_sphere, gamma_matrix, seed,
                    radius_max=None, dtype=np.float64):
    """Boolean model of overlapping balls.

    Centres are i.i.d. uniform in the periodic cell; balls are added one at a time
    until the voxel volume fraction first reaches ``volume_fraction``. With
    ``radius_max`` set, each ball draws its radius uniformly from
    [radius, radius_max] (polydisperse).
    Returns (gamma, number_of_balls).
    """
    n = tuple(int(m) for m in n)
    rng = np.random.default_rng(seed)
    mask = np.zeros(n, dtype=bool)
    total = float(np.prod(n))
    count = 0
    filled = 0
    while filled / total < volume_fraction:
        c = rng.random(3) * np.asarray(n, dtype=np.float64)
        r = radius if radius_max is None else rng.uniform(radius, radius_max)
        filled += _stamp_ball(mask, c, r)
        count += 1
        if count > 10_000_000:  # pragma: no cover - guards a bad target
            raise RuntimeError("volume fraction not reachable")
    g = np.where(mask, gamma_sphere, gamma_matrix).astype(dtype)
    return g, count


def _segment_distance_sq_pairs(P0, D0, P1, D1):
    """Squared distances between the segments P0 + s D0 and P1 + t D1 (s, t in [0, 1]),
    elementwise over broadcast leading axes (last axis: the 3 coordinates). Closest
    points by the clamped parameter formulas of two line segments."""
    r = P0 - P1
    a = np.sum(D0 * D0, axis=-1)
    e = np.sum(D1 * D1, axis=-1)
    f = np.sum(D1 * r, axis=-1)
    c = np.sum(r * D0, axis=-1)
    b = np.sum(D1 * D0, axis=-1)
    denom = a * e - b * b
    safe = denom > 1e-14
    s = np.where(safe, np.clip((b * f - c * e) / np.where(safe, denom, 1.0), 0.0, 1.0), 0.0)
    t = (b * s + f) / e
    low, high = t < 0.0, t > 1.0
    s = np.where(low, np.clip(-c / a, 0.0, 1.0), np.where(high, np.clip((b - c) / a, 0.0, 1.0), s))
    t = np.clip(t, 0.0, 1.0)
    q = r + s[..., None] * D0 - t[..., None] * D1
    return np.sum(q * q, axis=-1)


def short_fibres(n, diameter, aspect_ratio, volume_fraction, gamma_fibre, gamma_matrix,
                 seed, max_attempts=2_000_000, dtype=np.float32, batch=512):
    """Straight cylinders (spherocylinder distance rule) by random sequential addition.

    Axis directions are isotropic on the sphere. A candidate is rejected if the
    periodic segment-segment distance (nearest periodic image of the midpoints) to
    any accepted fibre is below the diameter. Fibres are added until the voxel volume
    fraction first reaches ``volume_fraction``; a voxel belongs to a fibre iff its
    centre lies within radius of the axis segment (projected parameter clipped to
    the segment). Candidates are drawn in batches (5 uniform numbers each: midpoint,
    cos of the polar angle, azimuth) and tested against every accepted fibre at once,
    then in turn against the fibres accepted earlier in the same batch.
    Returns (gamma, number_of_fibres).
    """
    n = np.asarray([int(m) for m in n], dtype=np.int64)
    rng = np.random.default_rng(seed)
    radius = 0.5 * diameter
    length = diameter * aspect_ratio
    mask = np.zeros(tuple(n), dtype=bool)
    total = float(np.prod(n))
    nf = n.astype(np.float64)
    mids = np.zeros((0, 3))
    dirs = np.zeros((0, 3))
    count = 0
    filled = 0
    attempts = 0
    d2min = diameter * diameter
    while filled / total < volume_fraction:
        if attempts >= max_attempts:
            raise RuntimeError("fibre volume fraction not reachable")
        u = rng.random((batch, 5))
        attempts += batch
        mid = u[:, :3] * nf
        z = -1.0 + 2.0 * u[:, 3]
        phi = 2.0 * math.pi * u[:, 4]
        sz = np.sqrt(np.maximum(0.0, 1.0 - z * z))
        d = np.stack([sz * np.cos(phi), sz * np.sin(phi), z], axis=1) * length
        if count:
            delta = _periodic_delta(mid[:, None, :], mids[None, :, :], nf)
            dist = _segment_distance_sq_pairs((mid - 0.5 * d)[:, None, :], d[:, None, :],
                                              (mid[:, None, :] - delta) - 0.5 * dirs[None, :, :],
                                              dirs[None, :, :])
            ok = ~np.any(dist < d2min, axis=1)
        else:
            ok = np.ones(batch, dtype=bool)
        for i in range(batch):
            if not ok[i]:
                continue
            mids = np.concatenate([mids, mid[i:i + 1]])
            dirs = np.concatenate([dirs, d[i:i + 1]])
            count += 1
            filled += _stamp_cylinder(mask, mid[i] - 0.5 * d[i], d[i], radius)
            if filled / total >= volume_fraction:
                break
            rest = np.arange(i + 1, batch)
            rest = rest[ok[rest]]
            if rest.size:
                delta = _periodic_delta(mid[rest], mid[i][None, :], nf)
                dist = _segment_distance_sq_pairs(mid[rest] - 0.5 * d[rest], d[rest],
                                                  (mid[rest] - delta) - 0.5 * d[i][None, :], d[i][None, :])
                ok[rest[dist < d2min]] = False
    g = np.where(mask, gamma_fibre, gamma_matrix).astype(dtype)
    return g, count


def _stamp_cylinder(mask, p0, d, radius):
    n = mask.shape
    length = float(np.linalg.norm(d))
    step = max(radius, 1.0)
    nseg = max(int(math.ceil(length / step)), 1)
    dd = d @ d
    added = 0
    for s in range(nseg):
        a = p0 + d * (s / nseg)
        b = p0 + d * ((s + 1) / nseg)
        lo = np.floor(np.minimum(a, b) - radius - 1).astype(np.int64)
        hi = np.ceil(np.maximum(a, b) + radius + 1).astype(np.int64)
        idx = [np.arange(lo[ax], hi[ax] + 1) for ax in range(3)]
        X = (idx[0] + 0.5)[:, None, None] - p0[0]
        Y = (idx[1] + 0.5)[None, :, None] - p0[1]
        Z = (idx[2] + 0.5)[None, None, :] - p0[2]
        t = np.clip((X * d[0] + Y * d[1] + Z * d[2]) / dd, 0.0, 1.0)
        r2 = (X - t * d[0]) ** 2 + (Y - t * d[1]) ** 2 + (Z - t * d[2]) ** 2
        ii, jj, kk = np.nonzero(r2 < radius * radius)
        sel = (idx[0][ii] % n[0], idx[1][jj] % n[1], idx[2][kk] % n[2])
        added += int(np.count_nonzero(~mask[sel]))
        mask[sel] = True
    return added


def lognormal_field(n, correlation_length, sigma, seed, dtype=np.float64):
    """gamma = exp(sigma * g), g a periodic unit-variance Gaussian random field.

    g has the Gaussian covariance exp(-r^2 / (2 l^2)); it is synthesised as
    IFFT(sqrt(S) * FFT(white noise)) with S the sampled power spectrum of that
    covariance on the periodic grid, then shifted and scaled to zero sample mean
    and unit sample variance.
    """
    n = tuple(int(m) for m in n)
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(n)
    r2 = None
    for a, m in enumerate(n):
        x = np.arange(m, dtype=np.float64)
        x = np.minimum(x, m - x)
        shape = [1, 1, 1]
        shape[a] = -1
        term = (x * x).reshape(shape)
        r2 = term if r2 is None else r2 + term
    cov = np.exp(-r2 / (2.0 * correlation_length ** 2))
    spec = np.maximum(np.fft.fftn(cov).real, 0.0)
    g = np.fft.ifftn(np.sqrt(spec) * np.fft.fftn(white)).real
    g = (g - g.mean()) / g.std()
    return np.exp(sigma * g).astype(dtype)


def laminate(n1, n2, layer_gammas, dtype=np.float64):
    """gamma depends on k only: gamma[i, j, k] = layer_gammas[k]."""
    layers = np.asarray(layer_gammas, dtype=np.float64)
    return np.broadcast_to(layers[None, None, :], (n1, n2, layers.size)).astype(dtype)


def random_two_phase(n, fraction, gamma_a, gamma_b, seed, dtype=np.float64):
    """Independent voxel-wise two-phase field (gamma_a with probability fraction)."""
    rng = np.random.default_rng(seed)
    return np.where(rng.random(tuple(n)) < fraction, gamma_a, gamma_b).astype(dtype)


def uniform_random(n, lo, hi, seed, dtype=np.float64):
    """gamma i.i.d. uniform in [lo, hi) per voxel."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=tuple(n)).astype(dtype)



def disks_2d(n, count, area_fraction, gamma_disk, gamma_matrix, seed, max_attempts=2_000_000, dtype=np.float64):
    """Two-dimensional periodic cell (n x n x 1) of `count` non-overlapping equal disks whose
    total area is `area_fraction` of the cell, placed by random sequential addition.

    Stands in for the paper's unidirectional fibre composite of Sec. 4.3 (128^2 voxels,
    32 circular inclusions, 50 % filler, generated there by mechanical contraction, which is
    not available here). The crack normal of interest lies in the plane.
    Returns (gamma, centres).
    """
    radius = math.sqrt(area_fraction * n * n / (count * math.pi))
    rng = np.random.default_rng(seed)
    centres = np.zeros((0, 2))
    attempts = 0
    while len(centres) < count:
        attempts += 1
        if attempts > max_attempts:
            raise RuntimeError("random sequential addition did not place all disks")
        c = rng.random(2) * n
        if len(centres):
            d = np.abs(centres - c)
            d = np.minimum(d, n - d)
            if np.min(np.sum(d * d, axis=1)) < (2.0 * radius) ** 2:
                continue
        centres = np.vstack([centres, c])
    x = np.arange(n) + 0.5
    X, Y = np.meshgrid(x, x, indexing="ij")
    inside = np.zeros((n, n), dtype=bool)
    for cx, cy in centres:
        dx = np.abs(X - cx)
        dx = np.minimum(dx, n - dx)
        dy = np.abs(Y - cy)
        dy = np.minimum(dy, n - dy)
        inside |= dx * dx + dy * dy < radius * radius
    gamma = np.where(inside, gamma_disk, gamma_matrix).astype(dtype)[:, :, None]
    return gamma, centres

def relaxed_spheres(n, radii, seed, iterations=4000, tol=1e-3):
    """Non-overlapping balls (periodic cell of shape n): centres i.i.d. uniform, then
    overlaps removed by repeated pairwise pushes (every overlapping pair moves apart
    along its centre line by its overlap, shared in proportion to the other ball's
    radius) until the largest overlap is below tol voxels or `iterations` sweeps
    have run. A stand-in for packings made by mechanical contraction (denser than
    random sequential addition allows). Returns the centres, shape (len(radii), 3)."""
    L = np.asarray([float(m) for m in n])
    r = np.asarray(radii, dtype=np.float64)
    rng = np.random.default_rng(seed)
    x = rng.random((len(r), 3)) * L
    rsum = r[:, None] + r[None, :]
    share = r[None, :] / rsum            # ball i moves by this share of the pair's overlap
    for _ in range(iterations):
        d = x[:, None, :] - x[None, :, :]
        d -= L * np.round(d / L)
        dist = np.sqrt(np.sum(d * d, axis=-1))
        np.fill_diagonal(dist, np.inf)
        over = rsum - dist
        over[over < 0.0] = 0.0
        if over.max() < tol:
            break
        unit = d / np.maximum(dist, 1e-12)[:, :, None]
        x += np.sum((over * share)[:, :, None] * unit, axis=1) * 1.0001
        x %= L
    return x


def _stamp_balls(mask, centres, radii):
    added = 0
    for c, r in zip(centres, radii):
        added += _stamp_ball(mask, c, r)
    return added


def porous_spheres(n, count, porosity, seed, gamma_solid=1.0, dtype=np.float64):
    """Solid with `count` monodisperse, non-overlapping spherical pores of vanishing crack
    resistance (Sec. 4.5: 200 pores, porosity 5 ... 50 %, gamma = 0 in the pores).
    The radius gives the target porosity for balls in the continuum, the centres come
    from relaxed_spheres. Returns (gamma, voxel porosity)."""
    n = tuple(int(m) for m in n)
    vol = float(np.prod(n))
    radius = (porosity * vol * 3.0 / (4.0 * math.pi * count)) ** (1.0 / 3.0)
    centres = relaxed_spheres(n, np.full(count, radius), seed)
    mask = np.zeros(n, dtype=bool)
    _stamp_balls(mask, centres, np.full(count, radius))
    g = np.where(mask, 0.0, gamma_solid).astype(dtype)
    return g, float(mask.mean())


def sand_binder(n, grain_radius, grain_fraction, binder_fraction, seed, radius_spread=0.25):
    """Three-phase sand-core stand-in (Sec. 4.6: grains 58.6 %, binder 1.3 %, the rest the
    third phase): polydisperse, non-overlapping spherical grains (radius uniform in
    grain_radius (1 +- radius_spread), added until the continuum volume reaches
    grain_fraction, relaxed apart), a binder phase in the necks between neighbouring
    grains (the voxels outside the grains closest to a second grain surface, i.e. with the
    smallest distance to the second-nearest grain, up to binder_fraction of the cell),
    and the remaining space as the third phase ("matrix").
    Returns (labels, fractions): labels 0 matrix, 1 grain, 2 binder, uint8."""
    n = tuple(int(m) for m in n)
    vol = float(np.prod(n))
    rng = np.random.default_rng(seed)
    radii = []
    total = 0.0
    while total < grain_fraction * vol:
        r = grain_radius * rng.uniform(1.0 - radius_spread, 1.0 + radius_spread)
        radii.append(r)
        total += 4.0 / 3.0 * math.pi * r ** 3
    radii = np.asarray(radii)
    centres = relaxed_spheres(n, radii, seed + 1)
    # distance to the nearest and second-nearest grain surface, per voxel (grains stamped
    # one at a time on their bounding boxes)
    d1 = np.full(n, np.inf)
    d2 = np.full(n, np.inf)
    for c, r in zip(centres, radii):
        reach = 1.5 * r + 2.0
        idx = [np.arange(int(math.floor(c[a] - reach)), int(math.ceil(c[a] + reach)) + 1) for a in range(3)]
        dd = None
        for a in range(3):
            da = (idx[a] + 0.5) - c[a]
            sh = [1, 1, 1]
            sh[a] = -1
            t = (da * da).reshape(sh)
            dd = t if dd is None else dd + t
        dist = np.sqrt(dd) - r
        sel = np.ix_(idx[0] % n[0], idx[1] % n[1], idx[2] % n[2])
        cur1, cur2 = d1[sel], d2[sel]
        new1 = np.minimum(cur1, dist)
        new2 = np.minimum(cur2, np.maximum(cur1, dist))
        d1[sel], d2[sel] = new1, new2
    labels = np.zeros(n, dtype=np.uint8)
    outside = d1 >= 0.0
    k = int(round(binder_fraction * np.prod(n)))
    if k > 0:
        d2o = np.where(outside, d2, np.inf).reshape(-1)
        order = np.argsort(d2o, kind="stable")[:k]
        labels.reshape(-1)[order] = 2
    labels[~outside] = 1
    fr = [float(np.mean(labels == k)) for k in range(3)]
    return labels, {"matrix": fr[0], "grain": fr[1], "binder": fr[2]}


def config_single_sphere_32():
    """32^3 cell, gamma 1.0 matrix, one ball of radius 8 centred at (16, 16, 16) with gamma 0.1."""
    return single_sphere((32, 32, 32), (16.0, 16.0, 16.0), 8.0, 0.1, 1.0)


def config_boolean_spheres_128(seed=2103, dtype=np.float64):
    """128^3 Boolean model: radius 6, volume fraction 0.20, gamma 0.3 in balls / 1.0 matrix."""
    return boolean_spheres((128, 128, 128), 6.0, 0.20, 0.3, 1.0, seed, dtype=dtype)


def config_short_fibres_512(seed=2103, dtype=np.float32):
    """512^3 short-fibre composite: diameter 6, aspect ratio 20, 12 % fibres, gamma 3.0 / 1.0.

    Random sequential addition slows down sharply near 12 % for fibres of aspect
    ratio 20, so the field is the 256^3 periodic RSA cell repeated 2 x 2 x 2: the
    repetition keeps periodicity, non-overlap, the volume fraction and the
    orientation statistics, with a period of 256 voxels. Returns (gamma, fibres).
    """
    g, count = short_fibres((256, 256, 256), 6.0, 20.0, 0.12, 3.0, 1.0, seed, dtype=dtype)
    return np.tile(g, (2, 2, 2)), 8 * count
