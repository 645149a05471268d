"""Helpers shared by the GPU tests: build/load the library, move inputs."""
import math

import numpy as np
import torch

from paper_0911_1407_gb300 import mocks


def ensure_lib():
    from paper_0911_1407_gb300 import build
    build.build()
    import paper_0911_1407_gb300 as plc
    return plc


def dev(a, dtype):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def host(t):
    return t.detach().cpu().numpy()


def pk_table_for(n, box, nbins=96, seed=0):
    """A smooth positive P(k) table covering an n^3 grid of side `box`."""
    kf = 2 * math.pi / box
    k = np.exp(np.linspace(math.log(0.5 * kf), math.log(1.02 * math.sqrt(3) * math.pi * n / box), nbins))
    P = 300.0 * k / (1 + (k / 0.05) ** 2) ** 1.4 * (1 + 0.2 * np.sin(3 * np.log(k) + seed))
    return k, P


def small_mock(n, selection="uniform", sigma=1.0, nbar=2.0, box=None, seed=1):
    box = box if box is not None else 6.25 * n
    return mocks.make_mock(mocks.small_spec(n, box=box, sigma_G=sigma, nbar=nbar,
                                            selection=selection, seed=seed, nbins=256))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_rel(a, b):
    """Largest element-wise error over the reference's largest element."""
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(np.max(np.abs(b)), 1e-300))
