"""Seeded synthetic workloads (inputs only; no arithmetic of the method lives here).

Each generator returns plain numpy arrays and a dict of problem parameters.  The shapes and
distributions follow the paper's validation and scaling workloads (Sec. IV: single blobs and
pairs near walls; Sec. V.A: a dense sedimented layer of microrollers near one wall), replaced
by seeded random draws because the paper's configurations are not available:

* ``bw_small``    - N = 100 above one wall, box 64 x 64, z in [0, 12], heights U[1.5, 10],
                    forces N(0,1), no torques; grid 128^2 x 65, m = 6, beta = 10.2 (FP64 case).
* ``slit_16k``    - N = 16384 in a slit z in [0, 20], box 256^2, heights U[1.2, 18.8], forces
                    and torques N(0,1); grid 384^2 x 97, h = 2/3, m = 5 with Table I betas.
* ``rollers_1m``  - N = 2^20 microrollers above one wall, box 2048^2, z in [0, 8], heights
                    max(|N(1.6, 0.3)|, 1.05), force (0, 0, -1) (gravity) and torque (0, 1, 0)
                    on every particle; grid 3072^2 x 65, h = 2/3, m = 5 with Table I betas.

* ``batch_systems`` - independent systems of uneven size for batched and served products: N
                    log-uniform on [100, 50000], box side 4 sqrt(N), xy grid the 7-smooth size
                    nearest L / 0.6, nz drawn from {33, 65, 97}; bottom wall z in [0, 12] with
                    heights U[1.2, 10], slit z in [0, 20] with U[1.2, 18.8], open z in [0, 20]
                    with U[2, 18]; forces and torques N(0,1); m = 5 with Table I betas.

* ``serving_systems`` - the served population: systems drawn like ``batch_systems`` with the wall
                    mode cycling over open, bottom wall and slit (uniform over the three); requests
                    are drawn uniformly from the population so that plans stay resident.

* ``lanczos_layer`` - the Lanczos-convergence suspension of Sec. IV.C: a base cell of 2048
                    non-overlapping spheres (random sequential addition, centre distance >= 2 R_h)
                    in L = 128.8 R_h (area fraction 0.39) tiled r x r times in xy (N = 2048 r^2),
                    two layers of heights (half near 1.1 R_h, half near 2.2 R_h: the bimodal
                    profile of the scaling test, drawn here), box height H = 7.5 R_h, forces only,
                    Table III monopole grid (150 r)^2 x 19, m = 4, beta = 1.87 m; R_h = 1.

Seeds are 20221004 + the workload's index (1, 2, 3, 4, 5; 6 for the served population).
"""

import numpy as np

SEED_BASE = 20221004

# Table I of the paper (force and torque, m = 5): R_h/h, beta_M/m, beta_D/m
_T1_M5 = (1.560, 1.305, 2.232)


def _uniform_xy(rng, n, L):
    return rng.uniform(0.0, L, n), rng.uniform(0.0, L, n)


def bw_small(n=100, seed_offset=1):
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    L = 64.0
    x, y = _uniform_xy(rng, n, L)
    z = rng.uniform(1.5, 10.0, n)
    pos = np.stack([x, y, z], axis=1)
    F = rng.standard_normal((n, 3))
    params = dict(Lx=L, Ly=L, zmin=0.0, zmax=12.0, mode="bottom_wall", nx=128, ny=128, nz=65,
                  m_M=6, beta_M=10.2, m_D=0, beta_D=0.0, eta=1.0)
    return params, pos, F, None


def slit_16k(n=16384, seed_offset=2, nxy=384, L=256.0, nz=97):
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    x, y = _uniform_xy(rng, n, L)
    z = rng.uniform(1.2, 18.8, n)
    pos = np.stack([x, y, z], axis=1)
    F = rng.standard_normal((n, 3))
    T = rng.standard_normal((n, 3))
    m = 5
    params = dict(Lx=L, Ly=L, zmin=0.0, zmax=20.0, mode="slit", nx=nxy, ny=nxy, nz=nz,
                  m_M=m, beta_M=m * _T1_M5[1], m_D=m, beta_D=m * _T1_M5[2], eta=1.0)
    return params, pos, F, T


def rollers_1m(n=1 << 20, seed_offset=3, nxy=3072, L=2048.0):
    """Sedimented roller layer.  Smaller n/nxy/L give the same layer at reduced size (density
    n/L^2 and h = L/nxy are kept by the callers that shrink it)."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    x, y = _uniform_xy(rng, n, L)
    z = np.maximum(np.abs(rng.normal(1.6, 0.3, n)), 1.05)
    pos = np.stack([x, y, z], axis=1)
    F = np.zeros((n, 3))
    F[:, 2] = -1.0
    T = np.zeros((n, 3))
    T[:, 1] = 1.0
    m = 5
    params = dict(Lx=L, Ly=L, zmin=0.0, zmax=8.0, mode="bottom_wall", nx=nxy, ny=nxy, nz=65,
                  m_M=m, beta_M=m * _T1_M5[1], m_D=m, beta_D=m * _T1_M5[2], eta=1.0)
    return params, pos, F, T


def random_particles(params, n, seed, torques=True, margin=None):
    """Uniform random particles inside a given box, heights kept where the envelope is legal
    for the wall mode (at least alpha from an open boundary).  Forces/torques N(0,1)."""
    rng = np.random.default_rng(seed)
    h = params["Lx"] / params["nx"]
    a = 0.5 * max(params["m_M"], params.get("m_D", 0) or 0) * h
    zlo, zhi = params["zmin"], params["zmax"]
    if margin is None:
        margin = 0.0
    lo = zlo + (a if params["mode"] == "free" else 0.0) + margin
    hi = zhi - (a if params["mode"] in ("free", "bottom_wall") else 0.0) - margin
    pos = np.stack([rng.uniform(0, params["Lx"], n), rng.uniform(0, params["Ly"], n),
                    rng.uniform(lo, hi, n)], axis=1)
    F = rng.standard_normal((n, 3))
    T = rng.standard_normal((n, 3)) if torques else None
    return pos, F, T


def smooth7_sizes(limit):
    """All 2,3,5,7-smooth integers in [8, limit]."""
    out = []
    for a in range(0, 20):
        for b in range(0, 13):
            for c in range(0, 9):
                for d in range(0, 7):
                    v = 2 ** a * 3 ** b * 5 ** c * 7 ** d
                    if 8 <= v <= limit:
                        out.append(v)
    return sorted(set(out))


_DOMAINS = {"bottom_wall": (12.0, 1.2, 10.0), "slit": (20.0, 1.2, 18.8), "free": (20.0, 2.0, 18.0)}


def batch_systems(count=256, seed_offset=4, modes=("bottom_wall", "slit"), n_range=(100, 50000), nz_set=(33, 65, 97)):
    """Independent systems of uneven size: a list of (params, pos, F, T).  Modes alternate over
    `modes` (half bottom wall, half slit by default)."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    sizes = np.array(smooth7_sizes(8192))
    out = []
    m = 5
    for i in range(count):
        mode = modes[i % len(modes)]
        n = int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        L = 4.0 * np.sqrt(n)
        nxy = int(sizes[np.argmin(np.abs(sizes - L / 0.6))])
        nz = int(rng.choice(nz_set))
        zmax, zlo, zhi = _DOMAINS[mode]
        x, y = _uniform_xy(rng, n, L)
        z = rng.uniform(zlo, zhi, n)
        pos = np.stack([x, y, z], axis=1)
        F = rng.standard_normal((n, 3))
        T = rng.standard_normal((n, 3))
        params = dict(Lx=L, Ly=L, zmin=0.0, zmax=zmax, mode=mode, nx=nxy, ny=nxy, nz=nz,
                      m_M=m, beta_M=m * _T1_M5[1], m_D=m, beta_D=m * _T1_M5[2], eta=1.0)
        out.append((params, pos, F, T))
    return out


def serving_systems(count=64, seed_offset=6):
    """The served population: (params, pos, F, T) systems of the batch size distribution, wall mode
    free, bottom wall, slit in turn."""
    return batch_systems(count=count, seed_offset=seed_offset, modes=("free", "bottom_wall", "slit"))


def _rsa_layer(rng, n, L, heights, dmin, max_tries=200000):
    """n spheres placed one at a time at a uniform xy position (periodic box of side L) and a height
    drawn by heights(rng), rejected while closer than dmin to one already placed (random
    sequential addition: no overlaps, as in a suspension with steric repulsion)."""
    pos = np.empty((n, 3))
    k = 0
    for _ in range(max_tries):
        p = np.array([rng.uniform(0.0, L), rng.uniform(0.0, L), heights(rng)])
        if k:
            d = pos[:k] - p
            d[:, :2] -= L * np.round(d[:, :2] / L)
            if np.min(np.einsum("ij,ij->i", d, d)) < dmin * dmin:
                continue
        pos[k] = p
        k += 1
        if k == n:
            return pos
    raise RuntimeError("random sequential addition did not place every particle")


def lanczos_layer(reps=1, mode="bottom_wall", seed_offset=5, H=7.5):
    """Particle layer of the Lanczos convergence test, tiled reps x reps times in xy; returns
    (params, pos, W) with W the i.i.d. standard normal vector [N][3].  H = 9.1 with reps = 18 is the
    largest force-only system of the scaling test (663,552 particles, grid 2700^2 x 19)."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    L0, n0 = 128.8, 2048

    def heights(r):  # two layers
        return r.normal(1.1, 0.05) if r.uniform() < 0.5 else r.normal(2.2, 0.1)

    base = _rsa_layer(rng, n0, L0, heights, 2.0)
    base[:, 2] = np.clip(base[:, 2], 1.0, 3.0)
    tiles = [base + np.array([i * L0, j * L0, 0.0]) for j in range(reps) for i in range(reps)]
    pos = np.concatenate(tiles)
    L = reps * L0
    params = dict(Lx=L, Ly=L, zmin=0.0, zmax=H, mode=mode, nx=150 * reps, ny=150 * reps, nz=19, m_M=4,
                  beta_M=4 * 1.87, m_D=0, beta_D=0.0, eta=1.0)
    W = rng.standard_normal((len(pos), 3))
    return params, pos, W
