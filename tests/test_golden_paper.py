"""Numbers the paper prints (tests/golden/paper_numbers.json) against arithmetic
that follows from its own definitions."""
import json
import math
import os

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_memory_claims_are_complex128_footprints():
    """Sec. Conclusions: 25 qubits need 18 PB as a density matrix and ~500 MB as a
    statevector -- 4^25 and 2^25 complex128 entries."""
    assert abs(4 ** 25 * 16 / 1e15 - 18) / 18 < 0.01
    assert abs(2 ** 25 * 16 / 1e6 - 500) / 500 < 0.1


def test_eq2_at_the_conclusions_point():
    """Eq. 2 at n = 25, K = 1000 gives about 1e-3: the '0.001%' of Sec. Conclusions
    reads as Error = 0.001 (0.1%), recorded as a paper inconsistency."""
    e = GOLD["eq2_error_model"]
    err = e["alpha"] * math.exp(e["delta"] * 25 - e["mu"] * math.log(1000))
    assert 0.9e-3 < err < 1.2e-3


def test_fig2_probabilities_match_product_mode_table():
    p = 0.2
    pr = oracle.pauli_probs(oracle.make_noise(p2=p, twoq_mode=1), True).reshape(4, 4)
    assert abs(pr[0, 0] - (1 - p) ** 2) < 1e-15
    assert abs(pr[1:, 1:].sum() - p ** 2) < 1e-15
