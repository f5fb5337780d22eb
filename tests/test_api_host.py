"""Argument checks of the Python front end that run before any library call (no GPU).

The library writes ndof doubles through every output pointer it receives, so an
output buffer of the wrong size, type, layout or device must be refused on the
host rather than handed to a kernel.
"""
import numpy as np
import pytest
import torch

from paper_1806_01422_gb300.api import Sem


def fake(ndof=16, shape=(2, 2, 4)):
    s = Sem.__new__(Sem)          # no library handle: only the host-side checks run
    s.ndof, s.shape, s.device = ndof, shape, torch.device("cpu")
    return s


def test_output_buffers_are_checked_before_the_library_writes_them():
    s = fake()
    good = torch.zeros(16, dtype=torch.float64)
    assert s._out(good, "out") is good
    assert s._out(None, "out").shape == (2, 2, 4)
    with pytest.raises(TypeError):
        s._out(torch.zeros(16, dtype=torch.float32), "out")
    with pytest.raises(TypeError):
        s._out(np.zeros(16), "out")
    with pytest.raises(ValueError):
        s._out(torch.zeros(15, dtype=torch.float64), "out")
    with pytest.raises(ValueError):
        s._out(torch.zeros(32, dtype=torch.float64)[::2], "out")     # not contiguous
    with pytest.raises(ValueError):
        s._out(torch.zeros(16, dtype=torch.float64, device="meta"), "out")   # another device


def test_inputs_are_converted_or_refused():
    s = fake()
    t = s._dev(np.arange(16.0), "u")
    assert t.shape == (2, 2, 4) and t.dtype == torch.float64
    assert s._dev(torch.arange(32.0, dtype=torch.float64)[::2], "u").is_contiguous()
    with pytest.raises(TypeError):
        s._dev(torch.zeros(16, dtype=torch.float32), "u")
    with pytest.raises(ValueError):
        s._dev(np.zeros(15), "u")
    with pytest.raises(TypeError):
        s._dev([0.0] * 16, "u")
