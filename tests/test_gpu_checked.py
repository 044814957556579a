"""The checked build (-DZBUS_CHECKED): every index the kernels read from a
table is tested against its buffer before use and a bad one is recorded in a
check word instead of faulting (a stand-in for a memory checker, which may
not run on these machines).  Small and odd sizes of every form (one-bus
feeder, batches of 1, 7 and 129, partial phases, batched feeders, gradients,
Newton-Raphson) run through libzbus_checked.so in a child process: no check
may fire and the results must match the oracles."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_runs_clean():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14103_gb300 import build as B
    path = B.build(checked=True)
    env = dict(os.environ, ZBUS_LIB=path)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked ok" in r.stdout


def test_pipeline_gives_up_without_a_fault_and_recovers():
    """The checked build's lowered wait limit makes the tensor-core pipeline
    give up: zbus_last_device_status reports ZBUS_ERR_TIMEOUT, and the next
    ordinary solve in the same process matches the oracle (tests/giveup_run.py)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14103_gb300 import build as B
    path = B.build(checked=True)
    env = dict(os.environ, ZBUS_LIB=path)
    r = subprocess.run([sys.executable, os.path.join(HERE, "giveup_run.py")], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "giveup ok" in r.stdout


def test_normal_build_reports_itself():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14103_gb300 import zbus
    flag, word = zbus.zbus_checked_status()
    assert flag == 0 and word == 0
    # the wait limit is not settable outside the checked build
    assert zbus.lib().zbus_checked_set_wait(0) == 7
