"""Seeded synthetic inputs for the viscous-Burgers workloads.

This module only draws random numbers (numpy PCG64 via ``default_rng``) and
evaluates smooth periodic test fields at coordinates supplied by the caller.
It holds none of the spectral-element arithmetic: the node coordinates come
from whichever side (library or test checker) consumes the field.

Fields (all periodic on the box, shaped ``(d, G, .., G)`` with the last axis
the x_0 direction, component c the velocity along x_c):

* ``field_1d``: u = sin x + 0.1 sum_{k=1..4} a_k sin(k x + phi_k),
  a_k ~ N(0,1), phi_k ~ U(0, 2 pi), on [0, 2 pi).
* ``field_2d``: per component sum of 16 modes A_m |k_m|^-2 sin(2 pi k_m.x + phi_m)
  with integer wave vectors 1 <= |k|_inf <= 8, A_m ~ N(0,1), phi_m ~ U(0, 2 pi),
  scaled so max |u| = 1, on [0, 1)^2.
* ``field_3d``: per component sum over every integer k with 1 <= |k| <= kmax of
  |k|^(-11/6) sin(2 pi k.x + phi_k), phi_k ~ U(0, 2 pi) (energy spectrum ~ k^(-5/3)),
  scaled so max |u| = 1, on [0, 1)^3; evaluated separably through complex
  exponentials per axis.
* ``field_random``: i.i.d. N(0,1) nodal values (operator parity inputs).

Exact solutions of the PDE used as data for the inverse problems of Sec. 6.1:

* ``advection_diffusion_1d``: u = sum_{j=1..5} c_j sin(2 pi j (x - a t)) exp(-4 pi^2 j^2 nu t),
  the solution of u_t + a u_x = nu u_xx on the unit period (coefficients c_j ~ U(0.9, 1)
  from ``advection_diffusion_coefs``).
* ``cole_hopf_1d``: the Cole-Hopf solution of viscous Burgers
  u = 2 nu pi sin(pi x) e / (2 + e cos(pi x)), e = exp(-nu pi^2 t), period 2; and
  ``gaussian_bump`` = exp(-4 (x - 2)^2), the perturbation of its initial guess.
"""
import numpy as np

SEED_U0 = 1
SEED_UOBS = 2


def batch_seeds(k):
    """Seeds of batch instance k: (u0 seed, u_obs seed)."""
    return 1000 + 2 * k, 1001 + 2 * k


def batch_shapes(count=256, seed=4, E_choices=(8, 16, 24, 32, 48), N_choices=(5, 7, 9)):
    """Seeded uneven instance sizes: (E per side, order N) for each of `count` instances."""
    rng = np.random.default_rng(seed)
    return [int(e) for e in rng.choice(E_choices, count)], [int(n) for n in rng.choice(N_choices, count)]


def field_1d(x, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(4)
    phi = rng.uniform(0.0, 2.0 * np.pi, 4)
    u = np.sin(x).copy()
    for k in range(1, 5):
        u += 0.1 * a[k - 1] * np.sin(k * x + phi[k - 1])
    return u[None, :]


def field_2d(x, seed, modes=16, kmax=8):
    rng = np.random.default_rng(seed)
    X0 = x[None, :]   # varies along the last axis (x_0)
    X1 = x[:, None]   # varies along the first axis (x_1)
    out = np.zeros((2, x.size, x.size))
    for c in range(2):
        m = 0
        while m < modes:
            k = rng.integers(-kmax, kmax + 1, size=2)
            if max(abs(k[0]), abs(k[1])) < 1:
                continue
            A = rng.standard_normal()
            phi = rng.uniform(0.0, 2.0 * np.pi)
            kn2 = float(k[0] ** 2 + k[1] ** 2)
            out[c] += A / kn2 * np.sin(2.0 * np.pi * (k[0] * X0 + k[1] * X1) + phi)
            m += 1
    return out / np.max(np.abs(out))


def field_3d(x, seed, kmax=16):
    rng = np.random.default_rng(seed)
    r = np.arange(-kmax, kmax + 1)
    K0, K1, K2 = np.meshgrid(r, r, r, indexing="ij")
    kn = np.sqrt(K0 ** 2 + K1 ** 2 + K2 ** 2)
    sel = (kn >= 1) & (kn <= kmax)
    # per-axis exponentials e^{2 pi i k x}: (2 kmax + 1, G)
    ex = np.exp(2j * np.pi * r[:, None] * x[None, :])
    out = np.zeros((3, x.size, x.size, x.size))
    for c in range(3):
        phi = rng.uniform(0.0, 2.0 * np.pi, size=K0.shape)
        C = np.where(sel, kn, 1.0) ** (-11.0 / 6.0) * np.exp(1j * phi) * sel
        # f[z, y, x] = Im sum_{k0,k1,k2} C[k0,k1,k2] e0[k0, x] e1[k1, y] e2[k2, z]
        t = np.tensordot(C, ex, axes=([0], [0]))        # (k1, k2, x)
        t = np.tensordot(t, ex, axes=([0], [0]))        # (k2, x, y)
        t = np.tensordot(t, ex, axes=([0], [0]))        # (x, y, z)
        out[c] = np.transpose(t.imag, (2, 1, 0))
    return out / np.max(np.abs(out))


def field_random(dim, G, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((dim,) + (G,) * dim)


def workload_field(dim, x, seed):
    """The workload initial/observed field for dimension ``dim`` at axis coordinates x."""
    if dim == 1:
        return field_1d(x, seed)
    if dim == 2:
        return field_2d(x, seed)
    return field_3d(x, seed)


def advection_diffusion_coefs(seed, modes=5):
    return np.random.default_rng(seed).uniform(0.9, 1.0, modes)


def advection_diffusion_1d(x, t, coefs, nu, speed):
    u = np.zeros_like(x, dtype=np.float64)
    for j, c in enumerate(coefs, start=1):
        u += c * np.sin(2.0 * np.pi * j * (x - speed * t)) * np.exp(-4.0 * np.pi ** 2 * j * j * nu * t)
    return u[None, :]


def cole_hopf_1d(x, t, nu):
    e = np.exp(-nu * t * np.pi ** 2)
    return (2.0 * nu * np.pi * np.sin(np.pi * x) * e / (2.0 + e * np.cos(np.pi * x)))[None, :]


def gaussian_bump(x):
    return np.exp(-4.0 * (x - 2.0) ** 2)[None, :]
