"""Host logic of the autotuner: the cache key of a particle set (no GPU)."""
import numpy as np

import workloads


def test_signature_is_stable_and_sensitive():
    from paper_1110_0836_gb300 import tune
    w = workloads.shock_tube(5000, seed=2)
    s0 = tune.signature(w, 0.001, "fp32_mixed")
    assert s0 == tune.signature(workloads.shock_tube(5000, seed=2), 0.001, "fp32_mixed")
    assert s0 != tune.signature(w, 0.002, "fp32_mixed")       # skin
    assert s0 != tune.signature(w, 0.001, "fp64")             # precision
    w2 = workloads.shock_tube(5000, seed=2)
    w2.lam = w2.lam * 1.5                                      # lambda range
    assert s0 != tune.signature(w2, 0.001, "fp32_mixed")
    assert s0 != tune.signature(workloads.shock_tube(6000, seed=2), 0.001, "fp32_mixed")
    assert len(s0) == 16 and all(c in "0123456789abcdef" for c in s0)


def test_candidates_are_valid_plan_options():
    from paper_1110_0836_gb300 import tune
    assert tune.CANDIDATES[0] == dict(tile=128, schedule=0, cell_frac=1.0)   # the defaults first
    for c in tune.CANDIDATES:
        assert c["tile"] in (64, 128) and c["schedule"] in (0, 1) and 0 < c["cell_frac"] <= 1
    assert len({tuple(sorted(c.items())) for c in tune.CANDIDATES}) == len(tune.CANDIDATES)
