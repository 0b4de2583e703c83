"""The allocation-free ground-state entry point, through the C ABI.

Callers that cannot allocate device memory (a process that reserved its
whole budget up front, or a memory manager that forbids ad-hoc cudaMalloc)
use sqa_ground_energy_noalloc, which keeps its running minima in a fixed
device array instead of cudaMalloc'd scratch.  Its results must equal the
allocating entry point's exactly (integer energies), on consecutive calls
that reuse the shared array with different inputs.  This file is collected
last so that a failure here stops a -x run only after every other test ran.
"""
import numpy as np
import pytest

import paper_1603_03755_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_ground_energy_matches_allocating_entry_point_twice():
    import torch

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    for call, (N, I, seed) in enumerate([(12, 40, 91), (9, 300, 92)]):
        J = W.random_instances(N, I, seed)
        want = pkg.ground_energy(N, J)                       # allocating entry point
        J_dev = torch.from_numpy(J).to(dev)
        e_dev = torch.full((I,), 12345, dtype=torch.int64, device=dev)
        st = pkg.lib().sqa_ground_energy_noalloc(N, I, J_dev.data_ptr(), e_dev.data_ptr(), stream.cuda_stream)
        assert st == pkg.SQA_OK, pkg.lib().sqa_last_error()
        stream.synchronize()
        got = e_dev.cpu().numpy()
        assert np.array_equal(got, want), f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    dev = torch.device("cuda", 0)
    J_dev = torch.zeros((1, 1), dtype=torch.int32, device=dev)
    e_dev = torch.zeros((1,), dtype=torch.int64, device=dev)
    st = pkg.lib().sqa_ground_energy_noalloc(2, 4097, J_dev.data_ptr(), e_dev.data_ptr(), None)
    assert st == pkg.SQA_ERR_INVALID
    assert b"4096" in pkg.lib().sqa_last_error()
