"""Seeded synthetic workloads shaped like the paper's experiments.

Holds none of the method's arithmetic: it only draws cross sections, sources and
initial states on cell centres and names the angular rule each workload uses (each
side of a comparison builds that rule itself).  Both the CUDA path's tests / bench and
the oracle receive the same arrays from here.

Workloads (cell centres x_i = x0 + (i + 1/2) h; vacuum boundaries unless stated):

* ``slab_1d``        [0,1], 256 cells, S16 Gauss-Legendre, sigma_t = 1, sigma_s = 0.99,
                     rho0 = exp(-(x-0.5)^2/0.005), G = 0, c dt = 0.01, 100 steps.
* ``checkerboard``   [0,1]^2, 256^2, CL(32,8) hemisphere (128 directions), 8x8 blocks with
                     sigma_s = 100 where block (I+J) is even, else 0.01; sigma_a = 0.1;
                     G = 1 on |x-1/2|, |y-1/2| < 1/16; f0 = 0; c dt = 0.005, 200 steps.
* ``lognormal``      1024^2, 128 directions, sigma_s = exp(Z), Z a squared-exponential
                     Gaussian random field (correlation length 0.1, FFT synthesis on a 2x
                     periodic embedding, scaled to unit sample variance, then x std=2),
                     sigma_a = 0.05, rho0 = exp(-|x-c|^2/0.005), c = (1/2,1/2), G = 0,
                     c dt = 0.002, 500 steps.
* ``batched``        64 instances from seed 4: side N ~ U{128..512}, 64 or 128 directions,
                     log-normal sigma_s with std ~ U[0.5,3], pulse centre ~ U[0.2,0.8]^2,
                     sigma_a = 0.05, c dt = 0.005, 100 steps.
* ``diffusive_disc`` 2048^2, CL(32,16) hemisphere (256 directions), sigma_s = 1000 in the
                     disc |x-(1/2,1/2)| < 0.3, else 1; sigma_a = 0.01; centred pulse;
                     c dt = 0.001, 300 steps.
* ``two_material_slab``, ``isotropic_scattering``, ``variable_scattering``: the problems of
                     Sec. 4.1-4.3 with the paper's data (see each generator).

Every generator takes a size override so the same recipe yields small test cases.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    domain: tuple            # (x0, x1, y0, y1)
    quadrature: tuple        # ("gl", n) or ("cl_hemi", n_phi, n_vz)
    sigma_t: np.ndarray
    sigma_s: np.ndarray
    source: np.ndarray
    rho0: np.ndarray
    c_dt: float
    steps: int
    inflow: np.ndarray = field(default_factory=lambda: np.zeros(4))
    meta: dict = field(default_factory=dict)

    @property
    def ncell(self):
        return self.nx * self.ny

    @property
    def nv(self):
        q = self.quadrature
        return q[1] if q[0] == "gl" else q[1] * q[2] // 2


def _centres(n, lo=0.0, hi=1.0):
    h = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * h


def _grid(nx, ny):
    x = _centres(nx)
    y = _centres(ny)
    X, Y = np.meshgrid(x, y)        # [ny, nx], x fastest when raveled
    return X, Y


def gaussian_random_field(n, corr_len, std, rng):
    """Zero-mean field with squared-exponential covariance exp(-r^2 / (2 l^2)) on [0,1]^2,
    by FFT synthesis on a 2n x 2n periodic grid of spacing 1/n; returns the n x n corner
    scaled to sample mean 0 and sample standard deviation `std`."""
    m = 2 * n
    k = np.fft.fftfreq(m, d=1.0 / n) * 2.0 * np.pi
    KX, KY = np.meshgrid(k, k)
    spec = np.exp(-0.5 * corr_len ** 2 * (KX ** 2 + KY ** 2))
    noise = rng.standard_normal((m, m))
    z = np.real(np.fft.ifft2(np.fft.fft2(noise) * np.sqrt(spec)))[:n, :n]
    z = z - z.mean()
    return std * z / z.std()


def pulse(nx, ny, cx=0.5, cy=0.5, width=0.005):
    X, Y = _grid(nx, ny)
    return np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / width).ravel()


def slab_1d(n=256, steps=100, c_dt=0.01, n_dirs=16):
    x = _centres(n)
    return Workload("slab_1d", n, 1, (0.0, 1.0, 0.0, 1.0), ("gl", n_dirs),
                    sigma_t=np.ones(n), sigma_s=np.full(n, 0.99), source=np.zeros(n),
                    rho0=np.exp(-(x - 0.5) ** 2 / 0.005), c_dt=c_dt, steps=steps)


def checkerboard(n=256, steps=200, c_dt=0.005, blocks=8, quad=(32, 8), seed=None):
    X, Y = _grid(n, n)
    I = np.minimum((X * blocks).astype(int), blocks - 1)
    J = np.minimum((Y * blocks).astype(int), blocks - 1)
    ss = np.where((I + J) % 2 == 0, 100.0, 0.01).ravel()
    sa = 0.1
    G = ((np.abs(X - 0.5) < 1.0 / 16) & (np.abs(Y - 0.5) < 1.0 / 16)).astype(np.float64).ravel()
    return Workload("checkerboard", n, n, (0.0, 1.0, 0.0, 1.0), ("cl_hemi",) + tuple(quad),
                    sigma_t=ss + sa, sigma_s=ss, source=G, rho0=np.zeros(n * n), c_dt=c_dt,
                    steps=steps)


def lognormal(n=1024, steps=500, c_dt=0.002, std=2.0, corr_len=0.1, seed=3, quad=(32, 8),
              sigma_a=0.05, centre=(0.5, 0.5)):
    rng = np.random.default_rng(seed)
    z = gaussian_random_field(n, corr_len, std, rng)
    ss = np.exp(z).ravel()
    return Workload("lognormal", n, n, (0.0, 1.0, 0.0, 1.0), ("cl_hemi",) + tuple(quad),
                    sigma_t=ss + sigma_a, sigma_s=ss, source=np.zeros(n * n),
                    rho0=pulse(n, n, *centre), c_dt=c_dt, steps=steps,
                    meta=dict(seed=seed, std=std))


def batched(count=64, seed=4, n_range=(128, 512), steps=100, c_dt=0.005, scale=1.0):
    """`scale` shrinks every side (for tests); the draws do not depend on it."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        quad = (16, 8) if rng.random() < 0.5 else (32, 8)
        std = float(rng.uniform(0.5, 3.0))
        centre = tuple(rng.uniform(0.2, 0.8, size=2))
        sub = int(rng.integers(0, 2 ** 31 - 1))
        ns = max(8, int(round(n * scale)))
        w = lognormal(n=ns, steps=steps, c_dt=c_dt, std=std, seed=sub, quad=quad, centre=centre)
        w.name = f"batched[{b}]"
        out.append(w)
    return out


def diffusive_disc(n=2048, steps=300, c_dt=0.001, quad=(32, 16)):
    X, Y = _grid(n, n)
    inside = ((X - 0.5) ** 2 + (Y - 0.5) ** 2) < 0.3 ** 2
    ss = np.where(inside, 1000.0, 1.0).ravel()
    sa = 0.01
    return Workload("diffusive_disc", n, n, (0.0, 1.0, 0.0, 1.0), ("cl_hemi",) + tuple(quad),
                    sigma_t=ss + sa, sigma_s=ss, source=np.zeros(n * n), rho0=pulse(n, n),
                    c_dt=c_dt, steps=steps)


# The paper's own problems of Sec. 4 (their data only; each run uses the tolerances the paper
# states for it).  Time is c t with c = 1, so c_dt is the paper's time step.

def two_material_slab(dx=0.1, dt=10.0, steps=100, n_gl=6):
    """Sec. 4.1: [0, 11]; sigma_s = 0, sigma_a = 1 on [0, 1], sigma_s = 100, sigma_a = 0 on
    [1, 11]; f = 0 at t = 0; isotropic inflow 5 at x = 0, vacuum at x = 11."""
    n = int(round(11.0 / dx))
    x = _centres(n, 0.0, 11.0)
    ss = np.where(x < 1.0, 0.0, 100.0)
    sa = np.where(x < 1.0, 1.0, 0.0)
    return Workload("two_material_slab", n, 1, (0.0, 11.0, 0.0, 1.0), ("gl", n_gl),
                    sigma_t=ss + sa, sigma_s=ss, source=np.zeros(n), rho0=np.zeros(n),
                    c_dt=dt, steps=steps, inflow=np.array([5.0, 0.0, 0.0, 0.0]))


def isotropic_scattering(n=81, sigma_s=1.0, cfl=1.0, t_end=2.5, quad=(40, 6)):
    """Sec. 4.2: [-1, 1]^2, sigma_a = 0, G = (10 / pi) exp(-100 (x^2 + y^2)), zero inflow and
    initial state, dt = CFL dx, up to t = 2.5."""
    h = 2.0 / n
    x = _centres(n, -1.0, 1.0)
    X, Y = np.meshgrid(x, x)
    G = (10.0 / np.pi * np.exp(-100.0 * (X ** 2 + Y ** 2))).ravel()
    dt = cfl * h
    steps = int(np.ceil(t_end / dt - 1e-9))
    ss = np.full(n * n, float(sigma_s))
    return Workload("isotropic_scattering", n, n, (-1.0, 1.0, -1.0, 1.0), ("cl_hemi",) + tuple(quad),
                    sigma_t=ss.copy(), sigma_s=ss, source=G, rho0=np.zeros(n * n), c_dt=dt,
                    steps=steps, meta=dict(cfl=cfl))


def variable_scattering(n=81, cfl=1.0, t_end=2.5, quad=(40, 6), zeta=1e-2):
    """Sec. 4.3: [-1, 1]^2, sigma_s = 99.9 c^4 (c + sqrt 2)^2 (c - sqrt 2)^2 + 0.1 for
    c = |x| < 1, else 1; sigma_a = 0; G = 0; zero inflow; isotropic initial state
    exp(-|x|^2 / (4 zeta^2)) / (4 pi zeta^2); dt = CFL dx, up to t = 2.5."""
    h = 2.0 / n
    x = _centres(n, -1.0, 1.0)
    X, Y = np.meshgrid(x, x)
    c = np.sqrt(X ** 2 + Y ** 2)
    r2 = np.sqrt(2.0)
    ss = np.where(c < 1.0, 99.9 * c ** 4 * (c + r2) ** 2 * (c - r2) ** 2 + 0.1, 1.0).ravel()
    rho0 = (np.exp(-(X ** 2 + Y ** 2) / (4 * zeta ** 2)) / (4 * np.pi * zeta ** 2)).ravel()
    dt = cfl * h
    steps = int(np.ceil(t_end / dt - 1e-9))
    return Workload("variable_scattering", n, n, (-1.0, 1.0, -1.0, 1.0), ("cl_hemi",) + tuple(quad),
                    sigma_t=ss.copy(), sigma_s=ss, source=np.zeros(n * n), rho0=rho0, c_dt=dt,
                    steps=steps, meta=dict(cfl=cfl))


BY_NAME = dict(slab_1d=slab_1d, checkerboard=checkerboard, lognormal=lognormal,
               diffusive_disc=diffusive_disc, two_material_slab=two_material_slab,
               isotropic_scattering=isotropic_scattering, variable_scattering=variable_scattering)
