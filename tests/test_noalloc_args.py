"""Host-side argument checks of the allocation-free entry point: every
mismatch the library cannot see through raw addresses (host tensors, wrong
dtypes, short buffers, too few offsets) raises ValueError before any launch.
Runs on CPU: the device test is replaced by a predicate."""
import pytest
import torch

import paper_2205_03251_gb300 as gp


def _args(n=3, C=48):
    return dict(ops=torch.zeros(64, dtype=torch.uint8), off=torch.tensor([0, 3, 6, 9][:n + 1], dtype=torch.int64),
                x=torch.zeros(C), t=torch.zeros(C), consts=torch.zeros(251), values=torch.zeros(n, C),
                fitness=torch.zeros(n))


def _check(a, on_device=lambda tensor: True):
    return gp.check_noalloc_args(a["ops"], a["off"], a["x"], a["t"], a["consts"], a["values"], a["fitness"],
                                 on_device=on_device)


def test_valid_arguments_pass():
    assert _check(_args()) == 3


def test_host_tensors_are_rejected():
    with pytest.raises(ValueError, match="CUDA"):
        _check(_args(), on_device=lambda tensor: tensor.is_cuda)


@pytest.mark.parametrize("field,value,what", [
    ("ops", torch.zeros(64, dtype=torch.int32), "uint8"),
    ("ops", torch.zeros(60, dtype=torch.uint8), "16"),
    ("off", torch.tensor([0, 3, 6, 9], dtype=torch.int32), "int64"),
    ("off", torch.tensor([0], dtype=torch.int64), "n_trees"),
    ("off", torch.tensor([], dtype=torch.int64), "n_trees"),
    ("x", torch.zeros(48, dtype=torch.float64), "float32"),
    ("t", torch.zeros(47), "as many"),
    ("consts", torch.zeros(250), "251"),
    ("values", torch.zeros(3, 47), "n_trees x n_cases"),
    ("fitness", torch.zeros(2), "n_trees"),
    ("values", torch.zeros(48, 3).t(), "contiguous"),
    ("x", torch.zeros(0), "cases"),
    ("fitness", [0.0, 0.0, 0.0], "tensor"),
])
def test_each_mismatch_raises(field, value, what):
    a = _args()
    a[field] = value
    with pytest.raises(ValueError, match=what):
        _check(a)
