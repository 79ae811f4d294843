"""CPU checks of the Python binding's host logic (no context is created without a GPU)."""
import numpy as np
import pytest
import torch

from paper_1806_03095_gb300 import api


@pytest.mark.parametrize("arg,index", [(1, 1), (np.int64(4), 4), ("cuda:2", 2), (torch.device("cuda", 3), 3)])
def test_cuda_device_forms(arg, index):
    assert api.cuda_device(arg) == torch.device("cuda", index)


@pytest.mark.parametrize("arg", ["cpu", torch.device("cpu")])
def test_cuda_device_rejects_other_devices(arg):
    with pytest.raises(ValueError):
        api.cuda_device(arg)


@pytest.mark.skipif(torch.cuda.is_available(), reason="the failure path of a machine without a GPU")
def test_context_without_a_device_raises():
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        api.DGCNS((2, 2, 2), (0, 0, 0), (1, 1, 1), (1, 1, 1), 3, 5, 4)
