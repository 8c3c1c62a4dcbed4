"""Seeded test cases shared by the oracle tests and the GPU parity tests.

Each case is (mesh, kappa, leaf_max, eta1, eta2, m, eps).  The small sets are
chosen so that the directional code paths are exercised: with the paper's
eta1 = 10, eta2 = 1 and leaf 32 a 1280-triangle sphere has no admissible block
at kappa = 4, so the stress sets lower eta1 and the leaf size.
"""
import synth

CASES = {
    # name: (mesh level, kappa, leaf, eta1, eta2, m, eps)
    "plain1280": (3, 4.0, 32, 10.0, 1.0, 4, 1e-4),     # paper parameters, no admissible block
    "laplace1280": (3, 0.0, 32, 10.0, 1.0, 4, 1e-4),   # kappa = 0: H^2 case
    "lowfreq1280": (3, 4.0, 16, 10.0, 1.0, 4, 1e-4),   # admissible blocks, D = {0}
    "dir320": (2, 3.0, 8, 1.0, 4.0, 3, 1e-4),          # tiny, every admissible block directional
    "mixed1280": (3, 8.0, 16, 5.0, 2.0, 3, 1e-4),      # directional levels above D = {0} levels
    "dir1280": (3, 8.0, 8, 1.0, 2.0, 4, 1e-4),         # directional, levels 7-9
    "dir320m6": (2, 3.0, 8, 1.0, 4.0, 6, 1e-4),        # k = 216: weight stacks of 129-256 columns
    "dir320m5": (2, 3.0, 8, 1.0, 4.0, 5, 1e-4),        # k = 125: the headline's order, 65-128 column stacks
    "plain5120m5": (4, 8.0, 32, 10.0, 1.0, 5, 1e-4),   # paper parameters, kappa h as the 20480 workload;
                                                       # nearfield panels up to 5120 columns (several parts)
}


def mesh(name):
    level = CASES[name][0]
    return synth.icosphere(level)


def params(name):
    _, kappa, leaf, eta1, eta2, m, eps = CASES[name]
    return dict(kappa=kappa, leaf=leaf, eta1=eta1, eta2=eta2, m=m, eps=eps)
