"""The oracle's whole loop against a brute-force restatement of one sweep.

tests/bruteforce.py writes one synchronous sweep out from the reading of the
paper with nothing of the oracle's: codes from the Kuhn simplices under the
(value, index) order, floors by exact rational arithmetic, the target and
reference rule and each edit rule.  Iterating it until no vertex is distorted
must give the oracle's field after every sweep (its log) and at the end, for
HALVE, SNAP and BELOW-REFERENCE.
"""
import numpy as np
import pytest

import oracle
from tests import bruteforce as bf


def grids(seed, count):
    rng = np.random.default_rng(seed)
    for trial in range(count):
        ndim = 2 + trial % 2
        shape = tuple(int(s) for s in rng.integers(2, 6, size=ndim))
        f = rng.integers(0, 7, size=shape).astype(np.float32) / np.float32(8)
        xi = np.float32(rng.choice([0.05, 0.1, 0.3]))
        noise = rng.uniform(-1, 1, size=shape) * float(xi) * 0.999
        fhat = (f.astype(np.float64) + noise).astype(np.float32)
        yield f, fhat, xi


@pytest.mark.parametrize("rule", [oracle.RULE_HALVE, oracle.RULE_SNAP, oracle.RULE_BELOW])
def test_loop_equals_iterated_bruteforce_sweeps(rule):
    for f, fhat, xi in grids(5 + rule, 40):
        r = oracle.correct(f, fhat, xi, rule=rule, log_capacity=400)
        g = fhat.copy()
        k = 0
        while True:
            g2, distorted, targets, changed = bf.brute_sweep(f, g, xi, rule)
            assert r.sweep_log[k, 1] == distorted and r.sweep_log[k, 2] == targets
            if distorted == 0:
                break
            assert r.sweep_log[k, 3] == changed
            g = g2
            k += 1
            if changed == 0:
                break
        assert r.status == (oracle.OK if distorted == 0 else oracle.STUCK)
        assert r.sweeps == k
        assert np.array_equal(r.g.view(np.uint32), g.view(np.uint32))
