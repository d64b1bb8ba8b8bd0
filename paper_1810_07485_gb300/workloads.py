"""Seeded synthetic workloads for the batched and served forms, and initial
Ising configurations.

Only parameter and input draws live here (no part of any update's
arithmetic): chain sizes and temperatures for a batch of independent chains,
a Poisson stream of simulation requests, and random spin configurations for
the Swendsen-Wang lattice.  Benchmarks and tests draw from the same
generators.
"""
import numpy as np


def round_even(x):
    return max(2, int(round(x / 2.0)) * 2)


def batch_specs(n_chains, L_min=32, L_max=4096, U_min=0.25, U_max=4.0, seed=0):
    """n_chains independent S=1/2 chains: L log-uniform in [L_min, L_max]
    (even), beta = L * U with U log-uniform in [U_min, U_max], seeds 0..n-1."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_chains):
        L = round_even(np.exp(rng.uniform(np.log(L_min), np.log(L_max))))
        U = float(np.exp(rng.uniform(np.log(U_min), np.log(U_max))))
        out.append(dict(L=L, beta=L * U, S=0.5, J=1.0, seed=i))
    return out


def request_stream(n_requests, rate, L_min=64, L_max=65536, U_min=0.25, U_max=4.0, n_updates=50,
                   seed=0):
    """Poisson arrivals at `rate` per second; each request a chain with S in
    {1/2, 1} (equal odds), L log-uniform in [L_min, L_max] (even), beta = L*U
    with U log-uniform in [U_min, U_max], n_updates updates.  Returns a list
    of (arrival_time_s, spec)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        S = 0.5 if rng.random() < 0.5 else 1.0
        L = round_even(np.exp(rng.uniform(np.log(L_min), np.log(L_max))))
        U = float(np.exp(rng.uniform(np.log(U_min), np.log(U_max))))
        out.append((t, dict(L=L, beta=L * U, S=S, J=1.0, seed=1000 + i, n_updates=n_updates)))
    return out


def ising_spins(L, seed, up_fraction=0.5):
    """L x L spins in {0, 1} (row-major), each 1 with probability 1 - up_fraction."""
    rng = np.random.default_rng(seed)
    return (rng.random(L * L) >= up_fraction).astype(np.uint8)
