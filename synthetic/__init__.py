"""Seeded synthetic inputs for the solver workloads.

Shared by the oracle tests, the GPU parity tests and the benchmark.  It holds no solver
arithmetic: every function evaluates a closed-form field at coordinates the caller
supplies.  Random numbers come from NumPy's PCG64 with base seed 1612.

Workloads (each is a stand-in for the analytic problems of the paper's Sec. 7; no dataset
is involved):

* ``poisson_manufactured``: -Laplace(u) = g on the unit square with
  u* = sin(pi x) sin(2 pi y) + x^2 y.
* ``VarCoeffProblem``: the variable-coefficient operator of Eq. defA with coefficient
  fields built from seeded 8-mode Fourier series (c11, c22 = 1 + 0.5 tanh(s), c12 a
  scaled series kept uniformly elliptic, c1, c2 series, c = |series| >= 0), a smooth
  load g and Dirichlet data from u*.
* ``heat_initial``: sums of 20 seeded Gaussians (backward-Euler heat stepping, Sec. 7.6
  style), one member per seed offset.
"""
import numpy as np

BASE_SEED = 1612


def rng(offset=0):
    return np.random.Generator(np.random.PCG64(BASE_SEED + offset))


class FourierSeries:
    """s(x, y) = sum_j a_j cos(2 pi (k_j x' + l_j y') + phi_j) with (k_j, l_j) drawn from
    {0..3}^2 minus (0, 0), a_j ~ N(0, 1), phi_j ~ U[0, 2 pi); x', y' are the coordinates
    mapped to [0, 1] over ``box``.  Scaled so that max |s| = 1 on a 256 x 256 grid."""

    def __init__(self, gen, modes=8, kmax=3, box=(0.0, 0.0, 1.0, 1.0)):
        self.box = box
        kl = []
        while len(kl) < modes:
            k, l = gen.integers(0, kmax + 1, size=2)
            if k == 0 and l == 0:
                continue
            kl.append((int(k), int(l)))
        self.kl = np.array(kl, dtype=np.float64)
        self.a = gen.standard_normal(modes)
        self.phi = gen.uniform(0.0, 2.0 * np.pi, size=modes)
        t = np.linspace(0.0, 1.0, 256)
        X, Y = np.meshgrid(t, t)
        x0, y0, x1, y1 = box
        self.scale = 1.0
        self.scale = 1.0 / np.max(np.abs(self(x0 + (x1 - x0) * X, y0 + (y1 - y0) * Y)))

    def __call__(self, x, y):
        x0, y0, x1, y1 = self.box
        xs = (np.asarray(x, dtype=np.float64) - x0) / (x1 - x0)
        ys = (np.asarray(y, dtype=np.float64) - y0) / (y1 - y0)
        s = np.zeros(np.broadcast(xs, ys).shape)
        for (k, l), a, ph in zip(self.kl, self.a, self.phi):
            s = s + a * np.cos(2.0 * np.pi * (k * xs + l * ys) + ph)
        return self.scale * s


def u_star(x, y):
    """Manufactured solution u* = sin(pi x) sin(2 pi y) + x^2 y."""
    return np.sin(np.pi * x) * np.sin(2 * np.pi * y) + x * x * y


def poisson_manufactured(x, y):
    """(c11, c12, c22, c1, c2, c, g) at the given points for -Laplace(u*) = g."""
    z = np.zeros_like(np.asarray(x, dtype=np.float64))
    g = 5.0 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(2 * np.pi * y) - 2.0 * y
    return (z + 1.0, z, z + 1.0, z, z, z), g


class VarCoeffProblem:
    """Variable-coefficient operator on [0,1]^2 (seed offsets 0..6 of the base seed).
    ``perturbed=True`` adds 0.1 |s7| to c (a seventh series), for the adjoint workload's
    observation field."""

    def __init__(self, box=(0.0, 0.0, 1.0, 1.0), seed_offset=0):
        self.box = box
        self.s = [FourierSeries(rng(seed_offset + k), box=box) for k in range(8)]

    def coeffs(self, x, y, perturbed=False):
        s = self.s
        c11 = 1.0 + 0.5 * np.tanh(s[0](x, y))
        c22 = 1.0 + 0.5 * np.tanh(s[1](x, y))
        amp = 0.2
        c12 = amp * s[2](x, y)
        while np.min(c11 * c22 - c12 * c12) <= 0.1:
            amp *= 0.5
            c12 = amp * s[2](x, y)
        c1 = s[3](x, y)
        c2 = s[4](x, y)
        c0 = np.abs(s[5](x, y))
        if perturbed:
            c0 = c0 + 0.1 * np.abs(s[7](x, y))
        return (c11, c12, c22, c1, c2, c0)

    def load(self, x, y):
        return self.s[6](x, y)

    def dirichlet(self, x, y):
        return u_star(x, y)


def heat_initial_params(member=0, n_gauss=20):
    """(a, alpha, centres) of ensemble member ``member``: a_i ~ U(0.5, 1),
    alpha_i ~ U(50, 300), centres ~ U[0.1, 0.9]^2 (seed offset 1000 + member)."""
    gen = rng(1000 + member)
    a = gen.uniform(0.5, 1.0, n_gauss)
    al = gen.uniform(50.0, 300.0, n_gauss)
    c = gen.uniform(0.1, 0.9, (n_gauss, 2))
    return a, al, c


def heat_initial(x, y, member=0, n_gauss=20):
    """Sum of 20 Gaussians a_i exp(-alpha_i |x - x_i|^2) with the parameters of
    ``heat_initial_params``."""
    a, al, c = heat_initial_params(member, n_gauss)
    out = np.zeros(np.broadcast(np.asarray(x), np.asarray(y)).shape)
    for i in range(n_gauss):
        out = out + a[i] * np.exp(-al[i] * ((x - c[i, 0]) ** 2 + (y - c[i, 1]) ** 2))
    return out


def random_directions(shape, n=10, seed_offset=500):
    """n seeded unit-norm Gaussian directions of the given shape."""
    out = []
    for k in range(n):
        v = rng(seed_offset + k).standard_normal(shape)
        out.append(v / np.linalg.norm(v))
    return out


def smooth_directions(X, Y, n=10, seed_offset=700, fields=6):
    """n seeded smooth directions of shape (fields, *X.shape): each field is an 8-mode
    Fourier series at the given coordinates; each direction is scaled to unit 2-norm."""
    out = []
    for k in range(n):
        v = np.array([FourierSeries(rng(seed_offset + 16 * k + j))(X, Y) for j in range(fields)])
        out.append(v / np.linalg.norm(v))
    return out


def lshape_load_centre(seed_offset=300):
    """Seeded centre of the point load on the L-shaped domain [-1,1]^2 minus [0,1]x[-1,0]:
    uniform in the L, at distance > 0.1 from its boundary."""
    gen = rng(seed_offset)
    while True:
        x, y = gen.uniform(-1.0, 1.0, 2)
        in_l = not (x > 0.0 and y < 0.0)
        far = min(x + 1.0, 1.0 - x, y + 1.0, 1.0 - y) > 0.1
        if x > 0.0:
            far = far and y > 0.1
        if y < 0.0:
            far = far and x < -0.1
        if in_l and far:
            return float(x), float(y)


def point_load(x, y, centre, width=1e-3):
    """g = exp(-|x - centre|^2 / width^2) (a Gaussian point load of the given width)."""
    return np.exp(-((x - centre[0]) ** 2 + (y - centre[1]) ** 2) / width ** 2)


def plane_wave(x, y, kappa, theta=0.3):
    """u = sin(kappa (x cos(theta) + y sin(theta))): solves -Laplace(u) - kappa^2 u = 0."""
    return np.sin(kappa * (np.cos(theta) * x + np.sin(theta) * y))


def helmholtz_scattering(x, y, kappa=40.0):
    """The variable-coefficient Helmholtz problem of Sec. 7.2 at the given points:
    -Laplace(u) - kappa^2 (1 - b(x)) u = g with the scattering potential b a sum of two
    Gaussians (amplitude 1/2, exponent 200, centres (7/20, 6/10) and (6/10, 9/20)) and the
    Gaussian load g = exp(-300 |x - (1/4, 3/4)|^2).  Returns (coefficients, g); the
    Dirichlet data are zero (the section does not state them)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.zeros_like(x)
    b = 0.5 * np.exp(-200.0 * ((x - 0.35) ** 2 + (y - 0.6) ** 2)) + \
        0.5 * np.exp(-200.0 * ((x - 0.6) ** 2 + (y - 0.45) ** 2))
    g = np.exp(-300.0 * ((x - 0.25) ** 2 + (y - 0.75) ** 2))
    return (z + 1.0, z, z + 1.0, z, z, -kappa ** 2 * (1.0 - b)), g
