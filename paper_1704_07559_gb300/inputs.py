"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no lattice Boltzmann arithmetic: it only builds macroscopic fields
(density fluctuation, velocity, velocity gradient, body force) and arbitrary population
arrays from fixed seeds.  Both the CUDA path and the CPU oracle turn these fields into
populations with their own code.

Conventions: fields are float64 numpy arrays indexed [component, z, y, x] (2D: nz = 1);
node n sits at integer coordinate n; grad[a*d + b] = d u_a / d x_b.
"""
import numpy as np


def _coords(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def taylor_green_3d(n, u0=0.02, pressure=False):
    """3D Taylor-Green vortex on an n^3 periodic box, wavenumber k = 2 pi / n:
    u = u0 (sin kx cos ky cos kz, -cos kx sin ky cos kz, 0).
    pressure=True adds the inviscid pressure as drho = 3 p (cs^2 = 1/3, rho0 = 1).
    Returns drho (1 field), u (3 fields), grad_u (9 fields)."""
    k = 2.0 * np.pi / n
    x, y, z = _coords(n, n, n)
    sx, cx = np.sin(k * x), np.cos(k * x)
    sy, cy = np.sin(k * y), np.cos(k * y)
    sz, cz = np.sin(k * z), np.cos(k * z)
    u = np.stack([u0 * sx * cy * cz, -u0 * cx * sy * cz, np.zeros_like(x)])
    g = np.zeros((9,) + x.shape)
    g[0] = u0 * k * cx * cy * cz
    g[1] = -u0 * k * sx * sy * cz
    g[2] = -u0 * k * sx * cy * sz
    g[3] = u0 * k * sx * sy * cz
    g[4] = -u0 * k * cx * cy * cz
    g[5] = u0 * k * cx * sy * sz
    drho = np.zeros_like(x)
    if pressure:
        p = u0 * u0 / 16.0 * (np.cos(2 * k * x) + np.cos(2 * k * y)) * (np.cos(2 * k * z) + 2.0)
        drho = 3.0 * p
    return drho, u, g


def taylor_green_2d(nx, ny, nz=1, u0=0.02, plane="xy", pressure=True):
    """2D Taylor-Green vortex (an exact Navier-Stokes solution, decaying as exp(-2 nu k^2 t))
    in the given coordinate plane of an nx x ny x nz periodic box; k = 2 pi / n along the plane's
    axes (both axes of the plane must have the same length n).  In 2D lattices use plane 'xy', nz=1.
    Returns drho, u (3 or 2 fields: 2 when nz == 1 and plane == 'xy'), grad_u (9 or 4 fields)."""
    axes = {"xy": (0, 1), "yz": (1, 2), "xz": (0, 2)}[plane]
    x, y, z = _coords(nx, ny, nz)
    X = (x, y, z)
    dims = (nx, ny, nz)
    a, b = axes
    assert dims[a] == dims[b]
    k = 2.0 * np.pi / dims[a]
    d = 2 if (nz == 1 and plane == "xy") else 3
    sa, ca = np.sin(k * X[a]), np.cos(k * X[a])
    sb, cb = np.sin(k * X[b]), np.cos(k * X[b])
    u = np.zeros((d,) + x.shape)
    u[a] = u0 * sa * cb
    u[b] = -u0 * ca * sb
    g = np.zeros((d * d,) + x.shape)
    g[a * d + a] = u0 * k * ca * cb
    g[a * d + b] = -u0 * k * sa * sb
    g[b * d + a] = u0 * k * sa * sb
    g[b * d + b] = -u0 * k * ca * cb
    drho = np.zeros_like(x)
    if pressure:
        drho = 3.0 * (u0 * u0 / 4.0) * (np.cos(2 * k * X[a]) + np.cos(2 * k * X[b]))
    return drho, u, g


def abc_flow(n, u0=0.02):
    """Arnold-Beltrami-Childress flow with A = B = C = u0/sqrt(3) on an n^3 periodic box:
    u = (A sin kz + C cos ky, B sin kx + A cos kz, C sin ky + B cos kx), an exact Navier-Stokes
    solution (Beltrami, curl u = k u) decaying as exp(-nu k^2 t).  Returns drho (zero), u, grad_u."""
    k = 2.0 * np.pi / n
    A = B = C = u0 / np.sqrt(3.0)
    x, y, z = _coords(n, n, n)
    u = np.stack([A * np.sin(k * z) + C * np.cos(k * y), B * np.sin(k * x) + A * np.cos(k * z),
                  C * np.sin(k * y) + B * np.cos(k * x)])
    g = np.zeros((9,) + x.shape)
    g[1] = -C * k * np.sin(k * y)      # d ux / dy
    g[2] = A * k * np.cos(k * z)       # d ux / dz
    g[3] = B * k * np.cos(k * x)       # d uy / dx
    g[5] = -A * k * np.sin(k * z)      # d uy / dz
    g[6] = -B * k * np.sin(k * x)      # d uz / dx
    g[7] = C * k * np.cos(k * y)       # d uz / dy
    return np.zeros_like(x), u, g


def random_fourier(nx, ny, nz, kmax=8, rms=0.03, seed=4, device=None):
    """Divergence-free random velocity field: Fourier modes with 0 < |k| <= kmax (integer
    wavevectors of the periodic box), unit-variance complex Gaussian amplitudes projected onto
    the plane normal to k, summed on the grid points (the real part of sum_k a_k exp(i k.x)) and
    scaled to the requested rms speed (rms of |u| over the box).  The same seed gives the same
    field at every grid size whose Nyquist limit exceeds kmax.  The sum is evaluated as an
    inverse FFT of the mode amplitudes, on the CPU (numpy) or, with device set, on that torch
    device (returned as torch tensors there).  Returns drho (zero), u (3 fields)."""
    K, amp = random_fourier_modes(kmax, seed)
    # modes beyond a small grid's Nyquist limit alias exactly (e^{ikx} = e^{i(k mod n)x} on the
    # grid points), which the accumulation into the spectrum reproduces
    if device is None:
        spec = np.zeros((3, nz, ny, nx), dtype=np.complex128)
        for (kx, ky, kz), a in zip(K, amp):
            spec[:, kz % nz, ky % ny, kx % nx] += a
        u = np.real(np.fft.ifftn(spec, axes=(1, 2, 3))) * (nx * ny * nz)
        speed_rms = np.sqrt((u * u).sum(0).mean())
        return np.zeros((nz, ny, nx)), u * (rms / speed_rms)
    import torch

    spec = torch.zeros((3, nz, ny, nx), dtype=torch.complex128, device=device)
    idx = torch.tensor(np.stack([K[:, 2] % nz, K[:, 1] % ny, K[:, 0] % nx], axis=1), device=device)
    vals = torch.tensor(amp, dtype=torch.complex128, device=device)
    for c in range(3):
        spec[c].index_put_((idx[:, 0], idx[:, 1], idx[:, 2]), vals[:, c], accumulate=True)
    u = torch.fft.ifftn(spec, dim=(1, 2, 3)).real * (nx * ny * nz)
    del spec
    speed_rms = torch.sqrt((u * u).sum(0).mean())
    return torch.zeros((nz, ny, nx), dtype=torch.float64, device=device), u * (rms / speed_rms)


def random_fourier_modes(kmax=8, seed=4):
    """The (wavevector, amplitude) list behind random_fourier, for evaluating the same field on
    another device.  Returns K (m, 3) int and amp (m, 3) complex, before rms scaling."""
    rng = np.random.default_rng(seed)
    ks = np.arange(-kmax, kmax + 1)
    KX, KY, KZ = np.meshgrid(ks, ks, ks, indexing="ij")
    K = np.stack([KX.ravel(), KY.ravel(), KZ.ravel()], axis=1)
    kk = (K * K).sum(1)
    sel = (kk > 0) & (kk <= kmax * kmax)
    K = K[sel]
    amp = rng.normal(size=(len(K), 3)) + 1j * rng.normal(size=(len(K), 3))
    kn = K / np.sqrt((K * K).sum(1, keepdims=True))
    amp = amp - (amp * kn).sum(1, keepdims=True) * kn
    return K, amp


def channel_profile(nx, ny, nz, u_centre=0.1, noise=0.01, seed=2):
    """Channel initial field with walls at the y faces (halfway, at y = -1/2 and ny - 1/2):
    a parabola u_x = u_centre * 4 s (1 - s), s = (y + 1/2)/ny, plus seeded uniform noise of
    relative amplitude +-noise (times u_centre) on all three components.  Returns drho, u."""
    rng = np.random.default_rng(seed)
    x, y, z = _coords(nx, ny, nz)
    s = (y + 0.5) / ny
    u = np.zeros((3,) + x.shape)
    u[0] = u_centre * 4.0 * s * (1.0 - s)
    u += noise * u_centre * rng.uniform(-1.0, 1.0, size=u.shape)
    return np.zeros_like(x), u


def random_populations(q, shape, scale=1e-3, seed=0, base=None):
    """Arbitrary population arrays (q, *shape): base (e.g. lattice weights times a density
    fluctuation, or zero) plus seeded Gaussian noise of the given scale."""
    rng = np.random.default_rng(seed)
    f = rng.normal(scale=scale, size=(q,) + tuple(shape))
    if base is not None:
        f += np.asarray(base, dtype=np.float64).reshape((q,) + (1,) * len(shape))
    return f


def gaussian_force(d, shape, std=1e-5, seed=5):
    """Body-force field (d, *shape) with independent N(0, std^2) entries."""
    rng = np.random.default_rng(seed)
    return rng.normal(scale=std, size=(d,) + tuple(shape))
