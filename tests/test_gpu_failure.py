"""Failure detection without a GPU fault: a launch whose wall-clock bound runs
out stops by itself (every wait and loop in the kernels is bounded), reports
PERM_ETIMEOUT through the status word, and leaves the context usable."""
import pytest

import paper_2002_03000_gb300 as pg
from paper_2002_03000_gb300 import _native as nat
from tests.gpu_util import Run, torch_cuda

pytestmark = pytest.mark.gpu


def test_time_bound_stops_the_launch_and_the_context_stays_usable(tmp_path):
    torch_cuda()
    # a run of about 0.2 s under a 2 ms bound
    with Run(2, 512, 4096, 1, max_seconds=0.002) as r:
        with pytest.raises(pg.PermError) as ei:
            r.run(64)
        assert ei.value.code == nat.PERM_ETIMEOUT
        st = r.stats()
        assert st["status"] == nat.PERM_ETIMEOUT
        assert 0 < st["steps"]
        # a failed run is not checkpointed
        with pytest.raises(pg.PermError) as ei:
            r.save(str(tmp_path / "failed.ckpt"))
        assert ei.value.code == nat.PERM_ETIMEOUT
        assert not (tmp_path / "failed.ckpt").exists()
    # the device and the library carry on
    with Run(2, 64, 256, 1) as r2:
        r2.run(4)
        st = r2.stats()
        assert st["status"] == 0 and st["tours_finished"] == 256 * 4


def test_a_failed_run_resets_and_runs_again():
    torch_cuda()
    with Run(2, 256, 2048, 2, max_seconds=0.002) as r:
        with pytest.raises(pg.PermError):
            r.run(64)
        r.reset()                       # clears the status and every per-tour sum
        st = r.stats()
        assert st["status"] == 0 and st["steps"] == 0
