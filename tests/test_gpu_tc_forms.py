"""The two forms of the tensor-core engine (persistent warp-specialised, the default, and one tile
per CTA, CRV_TC_WS=0) run the same split-FP32 products in the same K order, so their curvelet
coefficients and round trips agree bitwise; both reconstruct within the mixed tolerance."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _built():
    sys.path.insert(0, os.path.dirname(HERE))
    import __graft_entry__ as g
    g.build()


def _run(tmp_path, ws, L, spin):
    path = str(tmp_path / f"r_{ws}_{L}_{spin}.npz")
    env = dict(os.environ, CRV_TC_WS=ws)
    subprocess.run([sys.executable, os.path.join(HERE, "tc_forms_worker.py"), path, str(L), str(spin)],
                   check=True, env=env, timeout=600)
    return np.load(path)


@pytest.mark.parametrize("L,spin", [(45, 0), (32, 2)])
def test_engine_forms_agree_bitwise(tmp_path, L, spin):
    a = _run(tmp_path, "1", L, spin)
    b = _run(tmp_path, "0", L, spin)
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
    m = a["map"]
    assert np.linalg.norm(a["out"] - m) / np.linalg.norm(m) < 1e-5
