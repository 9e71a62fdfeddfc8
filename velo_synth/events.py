"""Seeded synthetic VELO-like events (input generator only).

This module draws hits; it contains none of the track-finding arithmetic
(no embedding, no distances, no message passing, no components).  Both the
FP64 oracle and the CUDA library read its output, so it must stay free of
anything either side computes.

Detector model (Sec. 2 and Sec. 3 of the paper): 26 planes perpendicular to
the beam, no magnetic field, so tracks are straight lines; a track leaves at
most one hit per plane here (overlapping sensors are not modelled), a hit
survives with the plane efficiency, and tracks start at a primary vertex
whose z spread is about 45 mm (Sec. 5.1).  Noise hits are uniform in the
annulus area of a random plane.  The paper trains and evaluates on LHCb
full simulation (Sec. 4); that sample is not available, so these events
stand in for it with the sizes the paper quotes (5.3 vertices per event).

Hits of one event are stable-sorted by plane index; every event is seeded
by ``base_seed + event_index`` so an event is bit-identical whether it is
generated alone or inside a batch.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

N_PLANES = 26
Z_PLANES = np.linspace(-287.0, 750.0, N_PLANES)  # mm, ascending: plane index = z order
R_MIN, R_MAX = 5.1, 40.0  # mm, sensitive annulus


@dataclass(frozen=True)
class EventRecipe:
    """How one event is drawn.  ``n_pv``/``tracks_per_pv`` are Poisson means
    when the matching ``*_poisson`` flag is set, fixed counts otherwise."""
    n_pv: float = 1
    n_pv_poisson: bool = False
    tracks_per_pv: float = 20
    tracks_poisson: bool = False
    eta_range: tuple = (2.0, 5.0)
    pv_z_sigma: float = 45.0      # mm
    hit_efficiency: float = 0.98
    smear: float = 0.012          # mm, Gaussian on x and y
    noise_fraction: float = 0.05  # noise hits = round(fraction * signal hits)
    z_planes: tuple = field(default=tuple(Z_PLANES.tolist()))


@dataclass
class Batch:
    """A ragged batch in structure-of-arrays form.

    x, y, z      float32 [N]   hit coordinates (mm)
    plane        int8    [N]   plane index 0..25, non-decreasing inside each event
    particle_id  int32   [N]   event-local particle index, -1 for noise
    hit_offsets  int32   [B+1] hits of event b are [hit_offsets[b], hit_offsets[b+1])
    """
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    plane: np.ndarray
    particle_id: np.ndarray
    hit_offsets: np.ndarray

    @property
    def n_events(self) -> int:
        return int(self.hit_offsets.shape[0] - 1)

    @property
    def n_hits(self) -> int:
        return int(self.hit_offsets[-1])

    def event(self, b: int) -> "Batch":
        lo, hi = int(self.hit_offsets[b]), int(self.hit_offsets[b + 1])
        return Batch(self.x[lo:hi], self.y[lo:hi], self.z[lo:hi], self.plane[lo:hi],
                     self.particle_id[lo:hi], np.array([0, hi - lo], np.int32))


def make_event(recipe: EventRecipe, seed: int):
    """Draw one event; returns (x, y, z, plane, particle_id), plane-sorted."""
    rng = np.random.default_rng(seed)
    zp = np.asarray(recipe.z_planes, np.float64)
    n_planes = zp.shape[0]
    n_pv = int(rng.poisson(recipe.n_pv)) if recipe.n_pv_poisson else int(recipe.n_pv)
    pv_z = rng.normal(0.0, recipe.pv_z_sigma, size=n_pv)
    if recipe.tracks_poisson:
        n_tr = rng.poisson(recipe.tracks_per_pv, size=n_pv).astype(np.int64)
    else:
        n_tr = np.full(n_pv, int(recipe.tracks_per_pv), np.int64)
    T = int(n_tr.sum())
    tz0 = np.repeat(pv_z, n_tr)
    eta = rng.uniform(recipe.eta_range[0], recipe.eta_range[1], size=T)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=T)
    keep_u = rng.uniform(size=(T, n_planes))
    sx = rng.normal(0.0, recipe.smear, size=(T, n_planes))
    sy = rng.normal(0.0, recipe.smear, size=(T, n_planes))

    tan_theta = np.tan(2.0 * np.arctan(np.exp(-eta)))
    dz = zp[None, :] - tz0[:, None]                      # [T, planes]
    r_true = dz * tan_theta[:, None]
    ok = (dz > 0) & (r_true > R_MIN) & (r_true < R_MAX) & (keep_u < recipe.hit_efficiency)
    ti, pi = np.nonzero(ok)                              # row-major: track-major order
    x_sig = r_true[ti, pi] * np.cos(phi[ti]) + sx[ti, pi]
    y_sig = r_true[ti, pi] * np.sin(phi[ti]) + sy[ti, pi]
    n_sig = ti.shape[0]

    n_noise = int(round(recipe.noise_fraction * n_sig))
    npl = rng.integers(0, n_planes, size=n_noise)
    nr = np.sqrt(rng.uniform(R_MIN ** 2, R_MAX ** 2, size=n_noise))
    nphi = rng.uniform(0.0, 2.0 * np.pi, size=n_noise)

    x = np.concatenate([x_sig, nr * np.cos(nphi)])
    y = np.concatenate([y_sig, nr * np.sin(nphi)])
    plane = np.concatenate([pi, npl]).astype(np.int64)
    z = zp[plane]
    pid = np.concatenate([ti, np.full(n_noise, -1)]).astype(np.int32)
    order = np.argsort(plane, kind="stable")
    return (x[order].astype(np.float32), y[order].astype(np.float32), z[order].astype(np.float32),
            plane[order].astype(np.int8), pid[order])


def make_batch(recipe: EventRecipe, n_events: int, base_seed: int) -> Batch:
    """Concatenate ``n_events`` events seeded ``base_seed + b``."""
    parts = [make_event(recipe, base_seed + b) for b in range(n_events)]
    return concat_events(parts)


def concat_events(parts) -> Batch:
    counts = np.array([p[0].shape[0] for p in parts], np.int64)
    offs = np.zeros(len(parts) + 1, np.int64)
    np.cumsum(counts, out=offs[1:])
    if offs[-1] >= 2 ** 31:
        raise ValueError("batch exceeds int32 hit indexing")
    cat = (lambda i, dt: np.concatenate([p[i] for p in parts]).astype(dt)
           if parts else np.zeros(0, dt))
    return Batch(cat(0, np.float32), cat(1, np.float32), cat(2, np.float32), cat(3, np.int8),
                 cat(4, np.int32), offs.astype(np.int32))


def truth_edge_labels(particle_id: np.ndarray, plane: np.ndarray, src: np.ndarray,
                      dst: np.ndarray) -> np.ndarray:
    """Genuine-edge targets (Fig. 2 caption: successive hits of one particle).

    With one hit per particle per plane, an edge i->j is genuine iff both hits
    belong to the same particle (id >= 0) and no hit of that particle lies on
    a plane strictly between plane(i) and plane(j).  Indices are into the
    given per-hit arrays (batch-global ids work because particle ids are
    offset per event by the caller, see ``global_particle_ids``)."""
    pid_s, pid_d = particle_id[src], particle_id[dst]
    same = (pid_s == pid_d) & (pid_s >= 0)
    y = np.zeros(src.shape[0], np.float32)
    if not same.any():
        return y
    # hit planes per particle: genuine iff consecutive in the particle's plane order
    key = particle_id.astype(np.int64) * 64 + plane.astype(np.int64)
    valid = particle_id >= 0
    keys = np.sort(key[valid])
    idx = np.nonzero(same)[0]
    ks, kd = key[src[idx]], key[dst[idx]]
    pos_s = np.searchsorted(keys, ks)
    pos_d = np.searchsorted(keys, kd)
    y[idx[pos_d == pos_s + 1]] = 1.0
    return y


def global_particle_ids(batch: Batch) -> np.ndarray:
    """Particle ids made unique across the batch (noise stays -1)."""
    out = batch.particle_id.astype(np.int64).copy()
    base = 0
    for b in range(batch.n_events):
        lo, hi = int(batch.hit_offsets[b]), int(batch.hit_offsets[b + 1])
        seg = out[lo:hi]
        m = seg >= 0
        if m.any():
            mx = int(seg[m].max()) + 1
            seg[m] += base
            base += mx
    return out


def compact_particle_ids(batch: Batch) -> np.ndarray:
    """Event-local particle ids renumbered 0..P-1 in ascending order of the
    original id (noise stays -1), so every id is below the event's hit count."""
    out = np.full(batch.n_hits, -1, np.int32)
    for b in range(batch.n_events):
        lo, hi = int(batch.hit_offsets[b]), int(batch.hit_offsets[b + 1])
        seg = batch.particle_id[lo:hi]
        m = seg >= 0
        if m.any():
            out[lo:hi][m] = np.unique(seg[m], return_inverse=True)[1]
    return out


def drop_noise(batch: Batch) -> Batch:
    """The batch without its noise hits (particle id -1), order kept: the
    embedding is trained on events with noise removed (Sec. 5.1)."""
    keep = batch.particle_id >= 0
    counts = np.array([int(keep[batch.hit_offsets[b]:batch.hit_offsets[b + 1]].sum())
                       for b in range(batch.n_events)], np.int64)
    offs = np.zeros(batch.n_events + 1, np.int64)
    np.cumsum(counts, out=offs[1:])
    return Batch(batch.x[keep], batch.y[keep], batch.z[keep], batch.plane[keep],
                 batch.particle_id[keep], offs.astype(np.int32))
