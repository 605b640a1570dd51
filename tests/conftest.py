import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def small_problem():
    """The small parity workload (N=20,000, d=32, two shards) with its input PGs."""
    import oracle as O
    from synth import gen, pgbuild
    w = gen.make("small")
    graphs = pgbuild.build_all(w)
    return w, graphs, O.Problem.from_workload(w, graphs)
