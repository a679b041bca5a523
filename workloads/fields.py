"""Field recipes for the synthetic workloads (no solver arithmetic here).

Physical constants follow Table 1 ("tab:params") of the paper, with the ice
strength P* read as 27.5 kN/m^2 (the printed unit "N/m^2" is taken to be a
typo: with 27.5 N/m^2 the ice would be in free drift) and a Coriolis
parameter f_c = 1.46e-4 1/s treated explicitly (Section 3, footnote on the
explicit Coriolis term).

Recipes:
  * GRF(seed, ell): white noise N(0,1) on the N x N cell grid, filtered in
    Fourier space by sqrt(S(k)), S(k) = exp(-|k|^2 ell^2 / 2) (Gaussian
    covariance with correlation length ell, periodic FFT), then normalised to
    zero mean and unit sample variance.
  * h = clip(1 + 0.5 GRF(s), 0.1, 3) m;  A = clip(0.95 + 0.05 GRF(s+1), 0, 1).
  * wind: Rankine vortex, speed 15 r/R (r <= R), 15 R/r (r > R), R = 100 km,
    cyclonic tangent rotated 20 degrees inward; centre ~ U[0.25L, 0.75L]^2
    from seed s+2 (or a translating centre c0 + 10 m/s t (1,1)/sqrt(2)).
  * ocean: 0.1 m/s gyre (-sin(pi x/L) cos(pi y/L), cos(pi x/L) sin(pi y/L)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Constants:
    """Physics and regularisation constants of the momentum equation."""
    rho_ice: float = 900.0      # kg/m^3
    rho_a: float = 1.3          # kg/m^3
    rho_o: float = 1026.0       # kg/m^3
    Ca: float = 1.2e-3
    Co: float = 5.5e-3
    f_c: float = 1.46e-4        # 1/s (explicit)
    Pstar: float = 27500.0      # N/m^2
    C: float = 20.0
    e: float = 2.0
    delta_min: float = 2e-9     # 1/s


@dataclasses.dataclass
class Problem:
    """One implicit momentum step: grid, constants and input fields."""
    N: int
    L: float
    const: Constants
    h: np.ndarray        # (N, N) ice thickness [m]
    A: np.ndarray        # (N, N) concentration [-]
    wind: np.ndarray     # (N+1, N+1, 2) [m/s] at t_{n+1}
    ocean: np.ndarray    # (N+1, N+1, 2) [m/s]
    v_old: np.ndarray    # (N+1, N+1, 2) [m/s]
    dt: float = 1800.0

    @property
    def dx(self) -> float:
        return self.L / self.N

    @property
    def ndof(self) -> int:
        return 2 * (self.N + 1) ** 2


def gaussian_random_field(N: int, L: float, ell: float, seed: int) -> np.ndarray:
    """Periodic Gaussian random field on the N x N cell grid (zero mean, unit variance)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.standard_normal((N, N))
    k = 2.0 * np.pi * np.fft.fftfreq(N, d=L / N)
    kx, ky = np.meshgrid(k, k, indexing="xy")
    filt = np.exp(-0.25 * (kx * kx + ky * ky) * ell * ell)   # sqrt(S)
    field = np.real(np.fft.ifft2(np.fft.fft2(noise) * filt))
    field -= field.mean()
    sd = field.std()
    return field / sd if sd > 0 else field


def ice_fields(N: int, L: float, seed: int, ell: float = 50e3):
    """Thickness h and concentration A on cells, from two GRFs (seeds s, s+1)."""
    h = np.clip(1.0 + 0.5 * gaussian_random_field(N, L, ell, seed), 0.1, 3.0)
    A = np.clip(0.95 + 0.05 * gaussian_random_field(N, L, ell, seed + 1), 0.0, 1.0)
    return h, A


def node_coords(N: int, L: float):
    x = np.linspace(0.0, L, N + 1)
    X, Y = np.meshgrid(x, x, indexing="xy")     # [j, i]
    return X, Y


def rankine_vortex(N: int, L: float, centre, vmax: float = 15.0, R: float = 100e3,
                   inflow_deg: float = 20.0) -> np.ndarray:
    """Rankine vortex wind at the nodes, shape (N+1, N+1, 2)."""
    X, Y = node_coords(N, L)
    dx = X - centre[0]
    dy = Y - centre[1]
    r = np.hypot(dx, dy)
    speed = np.where(r <= R, vmax * r / R, vmax * R / np.maximum(r, 1e-300))
    rs = np.where(r > 0, r, 1.0)
    tx, ty = -dy / rs, dx / rs            # cyclonic tangent
    ix, iy = -dx / rs, -dy / rs           # inward radial
    th = math.radians(inflow_deg)
    ux = math.cos(th) * tx + math.sin(th) * ix
    uy = math.cos(th) * ty + math.sin(th) * iy
    w = np.stack([speed * ux, speed * uy], axis=-1)
    w[r == 0] = 0.0
    return w


def ocean_gyre(N: int, L: float, umax: float = 0.1) -> np.ndarray:
    """Divergence-free sinusoidal gyre at the nodes, shape (N+1, N+1, 2)."""
    X, Y = node_coords(N, L)
    px, py = np.pi * X / L, np.pi * Y / L
    return np.stack([-umax * np.sin(px) * np.cos(py),
                     umax * np.cos(px) * np.sin(py)], axis=-1)


def vortex_centre(L: float, seed: int, lo: float = 0.25, hi: float = 0.75):
    rng = np.random.Generator(np.random.PCG64(seed))
    return tuple(rng.uniform(lo * L, hi * L, size=2))


def make_problem(N: int, seed: int, L: float = 512e3, const: Constants | None = None,
                 dt: float = 1800.0, centre=None, v_old=None) -> Problem:
    """The standard synthetic step: GRF ice, Rankine-vortex wind, gyre ocean."""
    const = const or Constants()
    h, A = ice_fields(N, L, seed)
    c = centre if centre is not None else vortex_centre(L, seed + 2)
    wind = rankine_vortex(N, L, c)
    ocean = ocean_gyre(N, L)
    vo = np.zeros((N + 1, N + 1, 2)) if v_old is None else np.array(v_old, dtype=np.float64)
    return Problem(N=N, L=L, const=const, h=h, A=A, wind=wind, ocean=ocean,
                   v_old=vo, dt=dt)


def make_problem_q2(N: int, seed: int, L: float = 512e3, const: Constants | None = None,
                    dt: float = 1800.0, centre=None, v_old=None) -> Problem:
    """The standard synthetic step for Q2 velocity elements on N x N cells: the
    same cell fields as ``make_problem(N, seed)``, the node fields on the
    (2N+1)^2 Q2 nodes (spacing L / 2N)."""
    const = const or Constants()
    h, A = ice_fields(N, L, seed)
    c = centre if centre is not None else vortex_centre(L, seed + 2)
    wind = rankine_vortex(2 * N, L, c)
    ocean = ocean_gyre(2 * N, L)
    vo = np.zeros((2 * N + 1, 2 * N + 1, 2)) if v_old is None else np.array(v_old, dtype=np.float64)
    return Problem(N=N, L=L, const=const, h=h, A=A, wind=wind, ocean=ocean, v_old=vo, dt=dt)


def translating_centre(L: float, seed: int, t: float, speed: float = 10.0):
    """Vortex centre at time t for the translating-vortex trajectory."""
    c0 = vortex_centre(L, seed + 2, 0.2, 0.35)
    s = speed * t / math.sqrt(2.0)
    return (c0[0] + s, c0[1] + s)


def problem_one(N: int, L: float = 512e3) -> Problem:
    """The paper's Problem I (Section 5.2): single momentum solve from rest on
    (0, 512 km)^2 with concentration
        A = 1 - 0.5 exp(-800 |r|) - 0.4 exp(-90 |r1|) - 0.4 exp(-90 |r1 + 0.7|),
        r  = 0.04 - (x/1000 km - 0.25)^2 - (y/1000 km - 0.25)^2,
        r1 = 0.1 + (2x/1000 km)^2 - (2y/1000 km)       (linear in y as printed),
    thickness H = 2A (evaluated at cell centres), wind (5, 5) m/s, ocean 0,
    dt = 0.5 h, Delta_min = 2e-9, no Coriolis term."""
    const = Constants(f_c=0.0)
    xc = (np.arange(N) + 0.5) * (L / N)
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    xs, ys = X / 1e6, Y / 1e6
    r = 0.04 - (xs - 0.25) ** 2 - (ys - 0.25) ** 2
    r1 = 0.1 + (2 * xs) ** 2 - (2 * ys)
    A = 1.0 - 0.5 * np.exp(-800 * np.abs(r)) - 0.4 * np.exp(-90 * np.abs(r1)) - 0.4 * np.exp(-90 * np.abs(r1 + 0.7))
    A = np.clip(A, 0.0, 1.0)
    wind = np.zeros((N + 1, N + 1, 2))
    wind[..., 0], wind[..., 1] = 5.0, 5.0
    z = np.zeros((N + 1, N + 1, 2))
    return Problem(N=N, L=L, const=const, h=2.0 * A, A=A, wind=wind, ocean=z, v_old=z.copy(), dt=1800.0)


def problem_two_wind(N: int, t: float, L: float = 512e3) -> np.ndarray:
    """Wind of the paper's Problem II (Section 5.3) at time t [s]: a cyclone
    moving along the diagonal, out for 4 days and back for 4,
        v_a = omega v_max(t) R(alpha) (x - m(t)),
        omega = exp(-|x - m| / 100 km) / 50,
        v_max = -15 tanh((4 - t)(4 + t) / 2) m/s (t <= 4 d),
                 15 tanh((12 - t)(t - 4) / 2) m/s (t > 4 d),
        alpha = 72 (t <= 4 d) or 81 degrees, R(alpha) = [[c, s], [-s, c]],
        m_x = m_y = 256 km + 51.2 km/d t (t <= 4 d), 665.6 km - 51.2 km/d t,
    with t in days and x - m in km (so that |v_a| peaks at 15*100/(50 e)
    = 11 m/s at 100 km from the centre)."""
    td = t / 86400.0
    if td <= 4.0:
        vmax, alpha, m = -15.0 * math.tanh((4.0 - td) * (4.0 + td) / 2.0), math.radians(72.0), 256.0 + 51.2 * td
    else:
        vmax, alpha, m = 15.0 * math.tanh((12.0 - td) * (td - 4.0) / 2.0), math.radians(81.0), 665.6 - 51.2 * td
    X, Y = node_coords(N, L)
    dx_, dy_ = X / 1e3 - m, Y / 1e3 - m
    om = np.exp(-np.sqrt(dx_ * dx_ + dy_ * dy_) / 100.0) / 50.0
    c, s = math.cos(alpha), math.sin(alpha)
    w = np.empty((N + 1, N + 1, 2))
    w[..., 0] = om * vmax * (c * dx_ + s * dy_)
    w[..., 1] = om * vmax * (-s * dx_ + c * dy_)
    return w


def problem_two_ocean(N: int, L: float = 512e3) -> np.ndarray:
    """Ocean current of Problem II: 0.01 m/s (-1 + 2y/L, 1 - 2x/L)."""
    X, Y = node_coords(N, L)
    o = np.empty((N + 1, N + 1, 2))
    o[..., 0] = 0.01 * (-1.0 + 2.0 * Y / L)
    o[..., 1] = 0.01 * (1.0 - 2.0 * X / L)
    return o


def problem_two(N: int, L: float = 512e3, delta_min: float = 2e-9) -> Problem:
    """First momentum step of the paper's Problem II (Section 5.3): ice at
    rest, A = 1, H = 0.3 m + 0.005 m (sin(60 x / 1000 km) + sin(30 y / 1000 km))
    at cell centres, dt = 0.5 h, no Coriolis term, wind at t_1 = dt.
    Later steps change only the wind (``problem_two_wind``), v_old, and the
    transported A and H."""
    const = Constants(f_c=0.0, delta_min=delta_min)
    xc = (np.arange(N) + 0.5) * (L / N)
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    H = 0.3 + 0.005 * (np.sin(60.0 * X / 1e6) + np.sin(30.0 * Y / 1e6))
    A = np.ones((N, N))
    dt = 1800.0
    return Problem(N=N, L=L, const=const, h=H, A=A, wind=problem_two_wind(N, dt, L), ocean=problem_two_ocean(N, L),
                   v_old=np.zeros((N + 1, N + 1, 2)), dt=dt)


CONFIG_NAMES = {
    0: "svN FP64, 64x64 cells (8,450 DOF), one 1800 s step from rest",
    1: "svN FP64, 512x512 cells (526,338 DOF), 10 steps, translating vortex",
    2: "mixed precision, 2048x2048 cells (8,396,802 DOF), 5 steps",
    3: "ensemble of 64 instances, N in {128,256,512,1024}",
    4: "learned start, 256x256 training grid",
}


def config(idx: int, delta_min: float = 2e-9, N: int | None = None) -> Problem:
    """First step of the named synthetic workload (overridable grid size)."""
    const = dataclasses.replace(Constants(), delta_min=delta_min)
    if idx == 0:
        return make_problem(N or 64, seed=0, const=const)
    if idx == 1:
        n = N or 512
        return make_problem(n, seed=1, const=const,
                            centre=translating_centre(512e3, 1, 1800.0))
    if idx == 2:
        return make_problem(N or 2048, seed=2, const=const)
    raise ValueError("config index must be 0, 1 or 2 (ensembles are built by the caller)")
