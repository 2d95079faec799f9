"""The integer issue-rate probe behind the roofline's denominator (needs a
GPU): every kind returns a finite positive rate, and the two pipes together
issue more than the logic pipe alone."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_issue_probe_rates(cuda_lib):
    ap = cuda_lib
    r = [ap.int_issue_probe(k, 20000) for k in (0, 1, 2)]
    assert all(math.isfinite(v) and v > 0 for v in r), r
    assert r[2] > r[0], r
