"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks. Holds none of the method's arithmetic: only random fields and the
node values of the Landau density used as a solver-only right-hand side.
"""
import numpy as np


def noise_field(N, seed, mean=0.0, sigma=1.0):
    """i.i.d. normal node values, FP64, flattened x-fastest."""
    return np.random.default_rng(seed).normal(mean, sigma, size=N ** 3)


def landau_density_nodes(N, alpha=0.05, k=0.5):
    """1 + alpha * (cos k x + cos k y + cos k z) at the nodes x_i = i L / N."""
    L = 2.0 * np.pi / k
    x = np.arange(N) * (L / N)
    c = np.cos(k * x)
    return (1.0 + alpha * (c[None, None, :] + c[None, :, None] + c[:, None, None])).reshape(-1)


def landau_noise_rhs(N, seed, alpha=0.05, k=0.5, sigma=0.01):
    """Landau density at the nodes plus N(0, sigma^2) noise (a shot-noise stand-in)."""
    return landau_density_nodes(N, alpha, k) + noise_field(N, seed, 0.0, sigma)


def landau_noise_rhs_torch(N, seed, device, alpha=0.05, k=0.5, sigma=0.01):
    """Same recipe generated on the device (for grids too large to build on the host)."""
    import torch
    L = 2.0 * np.pi / k
    x = torch.arange(N, dtype=torch.float64, device=device) * (L / N)
    c = torch.cos(k * x)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    rho = torch.empty(N, N, N, dtype=torch.float64, device=device)
    rho.normal_(0.0, sigma, generator=g)
    rho += 1.0 + alpha * (c[None, None, :] + c[None, :, None] + c[:, None, None])
    return rho.reshape(-1)
