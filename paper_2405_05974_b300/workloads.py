"""The synthetic workloads: mechanism sizes, state distributions and seeds.

The sizes mirror the paper's three QSS-reduced mechanisms (13-4-CH4,
35-18-nC12H26, 55-33-nC7H16; Section 3.2) at the scale of the tiny,
hydrocarbon and large workloads used throughout this package.  Every input
is synthetic and seeded; see ``mechgen``.
"""
from .mechgen import MechConfig, StateConfig

MECHS = {
    # 9 transported + 3 QSS, 30 reversible reactions (5 third-body),
    # one 2-species coupled QSS group.
    "tiny": MechConfig(name="tiny_9_3_30", n_transported=9, n_qss=3, n_reactions=30,
                       n_third_body=5, n_troe=0, qss_groups=[2, 1], seed=0,
                       all_reversible=True, max_carbon=2),
    # 35 + 18 species, 268 reactions (40 third-body, 25 Troe falloff),
    # QSS groups of size <= 4.
    "hydrocarbon": MechConfig(name="hc_35_18_268", n_transported=35, n_qss=18,
                              n_reactions=268, n_third_body=40, n_troe=25,
                              qss_groups=[4, 3, 2, 2, 2, 1, 1, 1, 1, 1], seed=1,
                              max_carbon=4),
    # 53 + 35 species, 1000 reactions (120 third-body, 80 Troe, 10% duplicates),
    # one 6-species group, the others <= 3.
    "large": MechConfig(name="large_53_35_1000", n_transported=53, n_qss=35,
                        n_reactions=1000, n_third_body=120, n_troe=80,
                        qss_groups=[6, 3, 3, 3, 2, 2, 2, 2] + [1] * 12, seed=2,
                        dup_fraction=0.10, max_carbon=6),
}

STATES = {
    "tiny": StateConfig(T_range=(1000.0, 2500.0), P_range_atm=(1.0, 1.0), P_log_uniform=False,
                        dirichlet_alpha=0.5, seed=0),
    "hydrocarbon": StateConfig(T_range=(900.0, 2800.0), P_range_atm=(1.0, 40.0),
                               P_log_uniform=True, dirichlet_alpha=0.3,
                               near_pure_fraction=0.05, seed=101),
    "large": StateConfig(T_range=(700.0, 3000.0), P_range_atm=(1.0, 60.0), P_log_uniform=False,
                         dirichlet_alpha=0.2, seed=102),
    # implicit-step workload: hydrocarbon mechanism and state distribution
    "implicit": StateConfig(T_range=(900.0, 2800.0), P_range_atm=(1.0, 40.0),
                            P_log_uniform=True, dirichlet_alpha=0.3,
                            near_pure_fraction=0.05, seed=103),
}

NCELLS = {"tiny": 4096, "hydrocarbon": 1 << 20, "large": 1 << 20, "implicit": 1 << 20}
# compiler options per workload: the large mechanism's Jacobian is built as a
# prefix kernel and 4 column-group kernels (its single-kernel form takes far
# longer to compile than its parts do in parallel; 2, 3 and 4 groups time
# within 1 % of each other, 8 groups 7 % slower, and 4 compile fastest)
# every workload's artefact also carries the mixed-precision Jacobian
# kernels (jac32: the source term in FP64, the derivative terms in FP32) for
# the mixed-precision implicit step; the FP64 kernels are the same as without.
# The hydrocarbon mixed kernel is spill-latency bound: 128 registers (four
# blocks per SM) and 64 FP32 values in shared memory measured fastest on B300
# (2^20 cells: 49.4 ms, against 60.0 ms at 255 registers without slots; 5
# blocks / 76 slots 49.3 ms, 6 / 64 51.7 ms, 4 / 96 50.0 ms)
BUILD_OPTIONS = {"tiny": {"jac32": True},
                 "hydrocarbon": {"jac32": True, "jac32_slots": 64, "jac32_minblocks": 4},
                 "large": {"jac_parts": 4, "jac32": True}}


def build_options(key: str) -> dict:
    return dict(BUILD_OPTIONS.get(key, {}))


# workloads whose artefacts carry the mixed-precision Jacobian kernels
# (one kernel, or the prefix and column groups of a partitioned Jacobian)
MIXED_JACOBIAN = tuple(k for k, o in BUILD_OPTIONS.items() if o.get("jac32"))
IMPLICIT_DT = 1.0e-6
# A second implicit-step size at which plain Newton from the initial state
# converges in >= 95 % of the hydrocarbon cells (oracle: 96.6 % at 1e-11 s,
# 72 % at 1e-8 s, 32 % at 1e-6 s): the synthetic Dirichlet compositions put
# radicals at mol/m^3 levels, so the fastest chemical time scales are ~1e-11 s
# and a larger step must jump most cells close to equilibrium.
IMPLICIT_DT_CONVERGING = 1.0e-11

_cache = {}


def mechanism(key: str) -> dict:
    """The seeded mechanism dictionary of workload ``key`` (memoised)."""
    from .mechgen import generate_mechanism
    if key not in _cache:
        _cache[key] = generate_mechanism(MECHS[key])
    return _cache[key]
