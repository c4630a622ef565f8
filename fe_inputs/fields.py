"""Smooth and random synthetic fields, evaluated at caller-supplied points."""
import numpy as np

from .rng import uniform, randint


def uniform_vector(n, seed, tag=0x7EC, lo=-1.0, hi=1.0, start=0):
    """``n`` doubles uniform in [lo, hi): entries start .. start+n-1 of the seeded vector."""
    return uniform(seed, tag, n, lo, hi, start=start)


def _sinusoid_params(seed, nterm=8):
    """Wave vectors k in {-2..2}^3 minus 0, amplitudes U[-1,1], phases U[0, 2pi)."""
    ks = np.zeros((3, nterm, 3), dtype=np.int64)
    draw = 0
    for c in range(3):
        for m in range(nterm):
            while True:
                k = randint(seed, 0x51A, 3, -2, 2, start=3 * draw)
                draw += 1
                if np.any(k != 0):
                    ks[c, m] = k
                    break
    amp = uniform(seed, 0xA3F, 3 * nterm, -1.0, 1.0).reshape(3, nterm)
    phase = uniform(seed, 0xF4A, 3 * nterm, 0.0, 2.0 * np.pi).reshape(3, nterm)
    return ks, amp, phase


def sinusoid_displacement(points, seed, amplitude=0.05, nterm=8):
    """Vector field u_c(x) = amplitude * sum_m a_cm sin(2 pi k_cm . x + phi_cm) / nterm.

    ``points`` is float64 [npts][3]; returns float64 [npts][3] (component
    fastest, i.e. already in the interleaved dof layout of a 3-vector field).
    """
    ks, amp, phase = _sinusoid_params(seed, nterm)
    out = np.zeros((points.shape[0], 3), dtype=np.float64)
    for c in range(3):
        for m in range(nterm):
            arg = 2.0 * np.pi * (points @ ks[c, m].astype(np.float64)) + phase[c, m]
            out[:, c] += amp[c, m] * np.sin(arg)
    return amplitude * out / nterm


def grf_fourier_features(points, seed, corr_len=0.1, nfeat=1024):
    """Gaussian random field sample by random Fourier features.

    f(x) = sqrt(2/nfeat) * sum_j cos(omega_j . x + b_j), omega_j ~ N(0, corr_len^-2 I),
    b_j ~ U[0, 2 pi): a stationary field with squared-exponential covariance of
    length ``corr_len`` (Rahimi and Recht, 2007).  Normal draws use Box-Muller.
    """
    u1 = uniform(seed, 0x6A1, 3 * nfeat, 0.0, 1.0)
    u2 = uniform(seed, 0x6A2, 3 * nfeat, 0.0, 1.0)
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    omega = (z / corr_len).reshape(nfeat, 3)
    b = uniform(seed, 0x6A3, nfeat, 0.0, 2.0 * np.pi)
    out = np.zeros(points.shape[0], dtype=np.float64)
    chunk = 4096
    for s in range(0, nfeat, chunk):
        e = min(nfeat, s + chunk)
        for j in range(s, e):
            out += np.cos(points @ omega[j] + b[j])
    return np.sqrt(2.0 / nfeat) * out


def grf_lattice(m, seed, corr_len=0.1, nfeat=256):
    """Gaussian random field on the m^3 equispaced lattice of the unit cube.

    Same random Fourier features as ``grf_fourier_features``; on a tensor
    lattice cos(w.x + b) is the real part of a product of three 1D complex
    exponentials, so the field is one complex matrix product:
    f[k, j, i] = Re sum_f c_f E2[f, k] E1[f, j] E0[f, i].  Returned flat with
    i fastest (lattice point i + m j + m^2 k).
    """
    u1 = uniform(seed, 0x6A1, 3 * nfeat, 0.0, 1.0)
    u2 = uniform(seed, 0x6A2, 3 * nfeat, 0.0, 1.0)
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    omega = (z / corr_len).reshape(nfeat, 3)
    b = uniform(seed, 0x6A3, nfeat, 0.0, 2.0 * np.pi)
    t = np.linspace(0.0, 1.0, m)
    E = [np.exp(1j * np.outer(omega[:, d], t)) for d in range(3)]  # [nfeat][m]
    c = np.sqrt(2.0 / nfeat) * np.exp(1j * b)
    T = (c[:, None, None] * E[1][:, :, None] * E[0][:, None, :]).reshape(nfeat, m * m)
    return np.real(E[2].T @ T).reshape(-1)
