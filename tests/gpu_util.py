"""Shared fixtures of the GPU tests: solver and oracle set-ups per workload."""
import functools

import numpy as np

from synth import draw_train, workload


@functools.lru_cache(maxsize=None)
def gpu_solver(name, **over):
    import __graft_entry__ as g
    g.build()
    import paper_2510_26180_gb300 as pkg
    w = workload(name, **over)
    return pkg.Solver(pkg.Problem.from_workload(w), draw_train(w)), w


@functools.lru_cache(maxsize=None)
def oracle_setup(name, processes=1, **over):
    from oracle.klecgc import Setup1D
    w = workload(name, **over)
    return Setup1D(w, processes=processes)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@functools.lru_cache(maxsize=None)
def oracle_setup2d(name, **over):
    from oracle.klecgc import Setup2D
    w = workload(name, **over)
    return Setup2D(w)


@functools.lru_cache(maxsize=None)
def oracle_setup_ac(name, **over):
    from oracle.klecgc import SetupAC1D
    w = workload(name, **over)
    return SetupAC1D(w)
