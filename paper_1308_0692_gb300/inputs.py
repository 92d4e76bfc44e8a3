"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

Holds random-number draws only -- none of the method's arithmetic -- so that
the CUDA path and the CPU oracle can be fed identical inputs without sharing
any solver code.
"""
from __future__ import annotations

import numpy as np

# seed of the batched parameter sweep (Kn/u_w over uneven grids)
BATCH_SEED = 20130803


def random_state(n: int, ncells: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """A random perturbation state h[a, cell] ~ N(0, scale^2), float64, SoA layout."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((n, ncells))


def random_cells(ncells: int, count: int, seed: int, include=()) -> np.ndarray:
    """Sorted distinct sample of cell indices (int64), always containing `include`."""
    rng = np.random.default_rng(seed)
    pick = rng.choice(ncells, size=min(count, ncells), replace=False)
    return np.unique(np.concatenate([pick, np.asarray(include, dtype=np.int64)])).astype(np.int64)


def batch_table(count: int = 512, seed: int = BATCH_SEED):
    """The batched sweep's instance table: half Couette channels with ny ~ U{64..512}, half
    cavities with side ~ U{64, 96, 128, 192, 256}; Kn log-uniform in [0.01, 10];
    u_w uniform in [0.005, 0.02].  Returns a list of dicts in draw order."""
    rng = np.random.default_rng(seed)
    out = []
    half = count // 2
    for i in range(count):
        geom = "couette" if i < half else "cavity"
        if geom == "couette":
            nx, ny = 1, int(rng.integers(64, 513))
        else:
            side = int(rng.choice([64, 96, 128, 192, 256]))
            nx = ny = side
        kn = float(10.0 ** rng.uniform(-2.0, 1.0))
        uw = float(rng.uniform(0.005, 0.02))
        out.append({"geom": geom, "nx": nx, "ny": ny, "kn": kn, "u_w": uw})
    return out
