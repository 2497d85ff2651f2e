"""Seeded synthetic trajectory workloads.

This module only draws inputs: aircraft-like trajectories sampled every 4 s
(the Mode-S radar period of Sec. 3.1), their wind measurements, and the
stress layouts of Sec. 4.2 (smoothed random walks, random points).  It holds
none of the nearest-neighbour arithmetic, so both the CUDA path and the CPU
oracle can take their inputs from it.

All arrays are produced with numpy's PCG64 generator from an explicit seed,
in float64, then cast once to float32.  Layout of every workload:

* ``xyzt``      float32 [N, 4]  x, y (km, tangent plane), z (km), t (s)
* ``wind``      float32 [N, 2]  measured wind (u, v) in m/s
* ``traj_off``  int64   [T + 1] trajectory boundaries; the points of
  trajectory i are rows traj_off[i]:traj_off[i+1], sorted by time
* ``flight``    int32   [N]     trajectory id of each row
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BOX_XY_KM = 2000.0
Z_MAX_KM = 12.0
T_SPAN_S = 21600.0
SAMPLE_DT_S = 4.0

# Seeds of the named workloads.
SEED_TINY = 0x7E01
SEED_MEDIUM = 0x7E02
SEED_PRECISION = 0x7E03
SEED_BATCHED = 0x7E04
SEED_LEARNED = 0x7E05
SEED_QUERY_SAMPLE = 0x5A00


@dataclass
class Workload:
    xyzt: np.ndarray
    wind: np.ndarray
    traj_off: np.ndarray
    flight: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.xyzt.shape[0])

    @property
    def n_traj(self) -> int:
        return int(self.traj_off.shape[0] - 1)


def _wind_field(rng: np.random.Generator, n_modes: int = 16, rms: float = 10.0):
    """Random smooth Fourier wind field: mean (20, 5) m/s plus n_modes plane
    waves in (x, y, z, t) with horizontal wavelengths 300-3000 km, vertical
    5-20 km and periods 3-24 h; amplitudes scaled to ``rms`` m/s total."""
    lam_h = np.exp(rng.uniform(math.log(300.0), math.log(3000.0), n_modes))
    ang = rng.uniform(0.0, 2.0 * math.pi, n_modes)
    lam_z = np.exp(rng.uniform(math.log(5.0), math.log(20.0), n_modes))
    sz = rng.choice([-1.0, 1.0], n_modes)
    per = np.exp(rng.uniform(math.log(3.0), math.log(24.0), n_modes)) * 3600.0
    st = rng.choice([-1.0, 1.0], n_modes)
    phi = rng.uniform(0.0, 2.0 * math.pi, n_modes)
    amp = rng.uniform(0.5, 1.5, n_modes)
    amp *= rms / math.sqrt(float(np.sum(amp * amp)))
    kx = 2.0 * math.pi / lam_h * np.cos(ang)
    ky = 2.0 * math.pi / lam_h * np.sin(ang)
    kz = sz * 2.0 * math.pi / lam_z
    om = st * 2.0 * math.pi / per

    def field(x, y, z, t):
        th = (np.outer(x, kx) + np.outer(y, ky) + np.outer(z, kz)
              + np.outer(t, om) + phi[None, :])
        u = 20.0 + (amp[None, :] * np.cos(th)).sum(axis=1)
        v = 5.0 + (amp[None, :] * np.sin(th)).sum(axis=1)
        return u, v

    return field


def _pack(x, y, z, t, u, v, lens, name) -> Workload:
    xyzt = np.stack([x, y, z, t], axis=1).astype(np.float32)
    wind = np.stack([u, v], axis=1).astype(np.float32)
    traj_off = np.zeros(len(lens) + 1, dtype=np.int64)
    traj_off[1:] = np.cumsum(np.asarray(lens, dtype=np.int64))
    flight = np.repeat(np.arange(len(lens), dtype=np.int32), lens)
    return Workload(np.ascontiguousarray(xyzt), np.ascontiguousarray(wind),
                    traj_off, flight, name)


def flights(n_flights: int, n_samples: int, seed: int, n_routes: int = 64,
            jitter_km: float = 0.05, name: str = "flights") -> Workload:
    """Aircraft on shared routes (Fig. 1: trajectories cluster along main
    routes).  Each route is a polyline of 3-5 random waypoints; each flight
    picks a route, a lateral offset N(0, 5 km), a cruise level U[8.5, 12] km
    that steps by +-0.6 km at each waypoint, a ground speed U[0.20, 0.26]
    km/s, a start position along the route and a start time, then is sampled
    every 4 s with N(0, jitter) position noise.  Rows are flight-major and
    time-sorted within each flight."""
    rng = np.random.default_rng(seed)
    routes = []
    for _ in range(n_routes):
        nw = int(rng.integers(3, 6))
        wp = rng.uniform(0.0, BOX_XY_KM, size=(nw, 2))
        seg = np.diff(wp, axis=0)
        seglen = np.linalg.norm(seg, axis=1)
        seglen = np.maximum(seglen, 1e-6)
        cum = np.concatenate([[0.0], np.cumsum(seglen)])
        routes.append((wp, seg / seglen[:, None], cum))
    field = _wind_field(rng)

    S = n_samples
    xs, ys, zs, ts = [], [], [], []
    for _ in range(n_flights):
        wp, dirs, cum = routes[int(rng.integers(0, n_routes))]
        lat = rng.normal(0.0, 5.0)
        speed = rng.uniform(0.20, 0.26)
        flen = speed * SAMPLE_DT_S * (S - 1)
        s0 = rng.uniform(0.0, max(cum[-1] - flen, 0.0))
        t0 = rng.uniform(0.0, T_SPAN_S - SAMPLE_DT_S * (S - 1))
        z0 = rng.uniform(8.5, Z_MAX_KM)
        steps = rng.choice([-0.6, 0.6], size=len(dirs))
        zl = np.clip(z0 + np.concatenate([[0.0], np.cumsum(steps[1:])]), 8.5, Z_MAX_KM)
        s = s0 + speed * SAMPLE_DT_S * np.arange(S)
        leg = np.clip(np.searchsorted(cum, s, side="right") - 1, 0, len(dirs) - 1)
        along = s - cum[leg]
        d = dirs[leg]
        nrm = np.stack([-d[:, 1], d[:, 0]], axis=1)
        p = wp[leg] + d * along[:, None] + nrm * lat
        z = zl[leg]
        p = p + rng.normal(0.0, jitter_km, size=p.shape)
        z = z + rng.normal(0.0, jitter_km, size=z.shape)
        xs.append(p[:, 0]); ys.append(p[:, 1]); zs.append(z)
        ts.append(t0 + SAMPLE_DT_S * np.arange(S))
    x = np.concatenate(xs); y = np.concatenate(ys)
    z = np.concatenate(zs); t = np.concatenate(ts)
    u, v = field(x, y, z, t)
    u = u + rng.normal(0.0, 1.0, size=u.shape)
    v = v + rng.normal(0.0, 1.0, size=v.shape)
    return _pack(x, y, z, t, u, v, [S] * n_flights, name)


def smoothed_random_walks(n_walks: int, n_samples: int, seed: int,
                          name: str = "srw") -> Workload:
    """Smoothed random walks (Sec. 4.2): constant speed ~0.23 km/s, heading
    whose rate of turn is itself a random walk, altitude drifting slowly;
    start point and time uniform in the box."""
    rng = np.random.default_rng(seed)
    field = _wind_field(rng)
    S = n_samples
    xs, ys, zs, ts = [], [], [], []
    for _ in range(n_walks):
        p = rng.uniform(0.0, BOX_XY_KM, size=2)
        z = rng.uniform(8.5, Z_MAX_KM)
        head = rng.uniform(0.0, 2.0 * math.pi)
        turn = np.cumsum(rng.normal(0.0, 0.002, size=S))
        hd = head + np.cumsum(turn)
        sp = 0.23 * SAMPLE_DT_S
        px = p[0] + np.concatenate([[0.0], np.cumsum(sp * np.cos(hd[1:]))])
        py = p[1] + np.concatenate([[0.0], np.cumsum(sp * np.sin(hd[1:]))])
        pz = np.clip(z + np.cumsum(rng.normal(0.0, 0.005, size=S)), 0.0, Z_MAX_KM)
        t0 = rng.uniform(0.0, T_SPAN_S - SAMPLE_DT_S * (S - 1))
        xs.append(px); ys.append(py); zs.append(pz)
        ts.append(t0 + SAMPLE_DT_S * np.arange(S))
    x = np.concatenate(xs); y = np.concatenate(ys)
    z = np.concatenate(zs); t = np.concatenate(ts)
    u, v = field(x, y, z, t)
    u = u + rng.normal(0.0, 1.0, size=u.shape)
    v = v + rng.normal(0.0, 1.0, size=v.shape)
    return _pack(x, y, z, t, u, v, [S] * n_walks, name)


def random_points(n_points: int, group: int, seed: int, name: str = "rand") -> Workload:
    """The pathological case of Sec. 4.2: points uniform in the box and in
    time, grouped at random into sets of ``group`` points (each set sorted by
    time so that it forms a valid 'trajectory')."""
    rng = np.random.default_rng(seed)
    field = _wind_field(rng)
    x = rng.uniform(0.0, BOX_XY_KM, n_points)
    y = rng.uniform(0.0, BOX_XY_KM, n_points)
    z = rng.uniform(0.0, Z_MAX_KM, n_points)
    t = rng.uniform(0.0, T_SPAN_S, n_points)
    lens = [group] * (n_points // group)
    if n_points % group:
        lens.append(n_points % group)
    off = np.concatenate([[0], np.cumsum(lens)])
    for i in range(len(lens)):
        sl = slice(off[i], off[i + 1])
        o = np.argsort(t[sl], kind="stable")
        x[sl] = x[sl][o]; y[sl] = y[sl][o]; z[sl] = z[sl][o]; t[sl] = t[sl][o]
    u, v = field(x, y, z, t)
    u = u + rng.normal(0.0, 1.0, size=u.shape)
    v = v + rng.normal(0.0, 1.0, size=v.shape)
    return _pack(x, y, z, t, u, v, lens, name)


def lattice(n_traj: int, n_samples: int, seed: int, side: int = 6,
            name: str = "lattice") -> Workload:
    """Tie-heavy input: walkers stepping on a small integer lattice with
    integer times, so that many pairs share exactly the same distance and
    duplicates of the same point occur."""
    rng = np.random.default_rng(seed)
    xs, ys, zs, ts = [], [], [], []
    for _ in range(n_traj):
        p = rng.integers(0, side, size=3).astype(np.float64)
        pts = [p.copy()]
        for _ in range(n_samples - 1):
            ax = int(rng.integers(0, 3))
            p[ax] = float(np.clip(p[ax] + rng.choice([-1.0, 0.0, 1.0]), 0, side - 1))
            pts.append(p.copy())
        pts = np.array(pts)
        t0 = float(rng.integers(0, 20))
        xs.append(pts[:, 0]); ys.append(pts[:, 1]); zs.append(pts[:, 2])
        ts.append(t0 + np.arange(n_samples, dtype=np.float64))
    x = np.concatenate(xs); y = np.concatenate(ys)
    z = np.concatenate(zs); t = np.concatenate(ts)
    u = rng.normal(0.0, 1.0, size=x.shape)
    v = rng.normal(0.0, 1.0, size=x.shape)
    return _pack(x, y, z, t, u, v, [n_samples] * n_traj, name)


# ---------------------------------------------------------------- named sets

SIGMA_DEFAULT = (1.0, 1.0, 10.0, 0.01)


def tiny() -> Workload:
    """200 flights x 50 samples = 10,000 points (k=8, 10-point segments)."""
    return flights(200, 50, SEED_TINY, name="tiny-10k")


def medium() -> Workload:
    """2,000 flights x 200 samples = 400,000 points (k=32, 20-point segments)."""
    return flights(2000, 200, SEED_MEDIUM, name="medium-400k")


def precision() -> Workload:
    """20,000 flights x 200 samples = 4,000,000 points (k=32)."""
    return flights(20000, 200, SEED_PRECISION, name="precision-4M")


def learned() -> Workload:
    """5,000 flights x 200 samples = 1,000,000 points (lag 1800 s)."""
    return flights(5000, 200, SEED_LEARNED, name="learned-1M")


def batched_windows(n_windows: int = 64, lo: float = 1e4, hi: float = 5e5,
                    seed: int = SEED_BATCHED, max_points: int | None = None):
    """Independent airspace/time windows with point counts log-uniform in
    [lo, hi] (each a whole number of 200-sample flights) and k drawn from
    {16, 32, 64}.  Returns a list of (Workload, k)."""
    rng = np.random.default_rng(seed)
    out = []
    for w in range(n_windows):
        nw = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        nf = max(1, int(round(nw / 200.0)))
        if max_points is not None:
            nf = max(1, min(nf, max_points // 200))
        k = int(rng.choice([16, 32, 64]))
        wl = flights(nf, 200, seed * 1000 + w, name=f"window{w}")
        out.append((wl, k))
    return out


def query_sample(n_total: int, n_sample: int, seed: int = SEED_QUERY_SAMPLE) -> np.ndarray:
    """Sorted, distinct query row ids drawn uniformly without replacement."""
    rng = np.random.default_rng(seed)
    n_sample = min(n_sample, n_total)
    return np.sort(rng.choice(n_total, size=n_sample, replace=False)).astype(np.int64)


def flight_split(wl: Workload, frac_test: float = 0.2, seed: int = 0xB0B0):
    """Split trajectory ids into train / held-out sets (held-out fraction
    ``frac_test``); returns boolean row masks (train, test)."""
    rng = np.random.default_rng(seed)
    T = wl.n_traj
    test_ids = rng.choice(T, size=max(1, int(round(frac_test * T))), replace=False)
    is_test = np.zeros(T, dtype=bool)
    is_test[test_ids] = True
    rows_test = is_test[wl.flight]
    return ~rows_test, rows_test
