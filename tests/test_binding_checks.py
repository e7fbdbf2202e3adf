"""The binding refuses output buffers the kernels could write past, before any call into the
library (host logic, no GPU)."""
import numpy as np
import pytest
import torch

from paper_2608_30239_gb300 import mcpd


def test_output_buffers_are_checked_before_a_launch():
    ok = torch.empty(10, dtype=torch.float64)     # right type and size, but in host memory
    with pytest.raises(TypeError, match="torch tensor"):
        mcpd._check_out(np.zeros(10), ok, 10, 0)
    with pytest.raises(TypeError, match="float64"):
        mcpd._check_out(torch.empty(10, dtype=torch.float32), ok, 10, 0)
    with pytest.raises(TypeError, match="contiguous"):
        mcpd._check_out(torch.empty(20, dtype=torch.float64)[::2], ok, 10, 0)
    with pytest.raises(ValueError, match="9 elements, 10 needed"):
        mcpd._check_out(torch.empty(9, dtype=torch.float64), ok, 10, 0)
    with pytest.raises(ValueError, match="the context is on cuda:0"):
        mcpd._check_out(ok, ok, 10, 0)           # host memory is not the context's device
