"""Memory-system probes behind the rooflines (gcc_probe_memory)."""
import math

import pytest

from paper_2406_10158_gb300 import engine as eng

pytestmark = pytest.mark.gpu


def test_probe_figures_are_physical():
    m = eng.gcc_probe_memory(0)
    for k, v in m.items():
        assert math.isfinite(v) and v > 0, (k, v)
    # a line in L2 answers sooner than one in HBM; one word's atomics are a
    # serial resource, distinct words are not
    assert m["l2_load_ns"] < m["hbm_load_ns"]
    assert m["occ_cycle_ns"] <= m["occ_cycle_busy_ns"]
    assert m["add_same_gops"] < m["cas_distinct_gops"]
    # a commit on one record costs at least one hand-off of its lock
    assert m["occ_cycle_ns"] > 0.5 * m["lock_handoff_ns"]
    assert m["contenders"] == 8 * m["sm_count"]
