"""The binding checks every tensor before its pointer crosses the C ABI.

The library receives bare device pointers and indexes them up to the problem's
length, so a tensor of the wrong type, layout, length or device would be read
or written out of bounds on the GPU.  These checks run on the host and need no
GPU: each wrong tensor must raise ValueError before any call is made.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1809_00828_gb300 import fcm  # noqa: E402


def test_wrong_dtype_raises():
    with pytest.raises(ValueError, match="dtype"):
        fcm._dev(torch.zeros(8, dtype=torch.float32), 8)


def test_non_contiguous_raises():
    t = torch.zeros(16, dtype=torch.float64)[::2]
    with pytest.raises(ValueError, match="contiguous"):
        fcm._dev(t, 8)


def test_wrong_length_raises():
    with pytest.raises(ValueError, match="elements"):
        fcm._dev(torch.zeros(7, dtype=torch.float64), 8)
    with pytest.raises(ValueError, match="multiple"):
        fcm._dev(torch.zeros(12, dtype=torch.float64), 8, multiple=True)
    with pytest.raises(ValueError, match="multiple"):
        fcm._dev(torch.zeros(0, dtype=torch.float64), 8, multiple=True)


def test_host_tensor_raises():
    with pytest.raises(ValueError, match="CUDA"):
        fcm._dev(torch.zeros(8, dtype=torch.float64), 8)
    with pytest.raises(ValueError, match="CUDA"):
        fcm._dev(torch.zeros(16, dtype=torch.float64), 8, multiple=True)


def test_not_a_tensor_raises():
    with pytest.raises(ValueError, match="torch tensor"):
        fcm._dev(np.zeros(8), 8)


def test_host_buffers_of_the_host_entry_points():
    with pytest.raises(ValueError):
        fcm._host_vec(np.zeros(8, dtype=np.float32), 8, "b")
    with pytest.raises(ValueError):
        fcm._host_vec(np.zeros(9), 8, "b")
    with pytest.raises(ValueError):
        fcm._host_vec(np.zeros(16)[::2], 8, "b")
    ro = np.zeros(8)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        fcm._host_vec(ro, 8, "out", writable=True)
    a = np.zeros(16)
    assert fcm._host_vec(a, 8, "b", multiple=True) is a


def test_choice_arguments_are_checked_before_any_call():
    # the named choices of the coarse correction and of the multi-level factors are validated in the
    # binding, before the object (here a stand-in) is used or the library is called
    dummy = object()
    with pytest.raises(ValueError):
        fcm.Solver.set_coarse_preconditioner(dummy, "amg")
    with pytest.raises(ValueError):
        fcm.Solver.set_coarse_storage(dummy, "bf16")
    with pytest.raises(ValueError):
        fcm.MLHPPlan.device_setup(dummy, stream=0, precision="fp16")
