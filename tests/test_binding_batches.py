"""Host-side argument checks of the binding's batch calls (no GPU): a stack of
batches must be a contiguous (nbatch, B, K) tensor with a matching
(nbatch, B, N) output, and is passed on as one (nbatch * B) x K matrix."""
import pytest
import torch

from paper_1106_0463_gb300 import _batch_args, _host_tensor


def test_stack_of_batches_is_passed_as_one_matrix():
    f, c = torch.zeros(3, 4, 9), torch.zeros(3, 4, 6)
    pf, pc, nb, B = _batch_args(f, c, 9, 6, torch.float32, _host_tensor, "_host")
    assert (nb, B) == (3, 4)
    assert pf.value == f.data_ptr() and pc.value == c.data_ptr()


@pytest.mark.parametrize("f,c", [
    (torch.zeros(4, 9), torch.zeros(3, 4, 6)),                      # f not a stack
    (torch.zeros(4, 3, 9).transpose(0, 1), torch.zeros(3, 4, 6)),   # f not contiguous
    (torch.zeros(3, 4, 9), torch.zeros(3, 5, 6)),                   # batch sizes differ
    (torch.zeros(3, 4, 8), torch.zeros(3, 4, 6)),                   # wrong K
    (torch.zeros(3, 4, 9, dtype=torch.float64), torch.zeros(3, 4, 6)),   # wrong type
    (torch.zeros(3, 4, 9), None),                                   # no output
])
def test_bad_stacks_are_rejected(f, c):
    with pytest.raises(ValueError):
        _batch_args(f, c, 9, 6, torch.float32, _host_tensor, "_host")
