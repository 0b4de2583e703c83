"""The allocation-free ground-state entry point, through the C ABI.

Callers that cannot allocate device memory (a process that reserved its
whole budget up front, or a memory manager that forbids ad-hoc cudaMalloc)
use sqa_ground_energy_noalloc, which keeps its running minima in a fixed
device array instead of cudaMalloc'd scratch.  Its results must equal the
allocating entry point's exactly (integer energies), on consecutive calls
that reuse the shared array with different inputs, including calls queued
one after another on one stream with no synchronisation between them.  This
file is collected last so that a failure here stops a -x run only after
every other test ran.
"""
import numpy as np
import pytest

import paper_1603_03755_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu


def _call(N, I, J_dev, e_dev, stream):
    return pkg.lib().sqa_ground_energy_noalloc(N, I, J_dev.data_ptr(), e_dev.data_ptr(), stream)


def test_noalloc_ground_energy_matches_allocating_entry_point_twice():
    import torch

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    # N = 12 and 9 walk one Gray-code chunk per thread; N = 20 splits the walk
    # into 2^2-state chunks over many threads
    for call, (N, I, seed) in enumerate([(12, 40, 91), (9, 300, 92), (20, 6, 93)]):
        J = W.random_instances(N, I, seed)
        want = pkg.ground_energy(N, J)                       # allocating entry point
        J_dev = torch.from_numpy(J).to(dev)
        e_dev = torch.full((I,), 12345, dtype=torch.int64, device=dev)
        st = _call(N, I, J_dev, e_dev, stream.cuda_stream)
        assert st == pkg.SQA_OK, pkg.lib().sqa_last_error()
        stream.synchronize()
        got = e_dev.cpu().numpy()
        assert np.array_equal(got, want), f"call {call}"


def test_noalloc_two_calls_queued_on_one_stream():
    """Two calls in a row on one stream, one synchronisation after both: the
    second call resets the shared minima only after the first has written its
    result, so each result is its own."""
    import torch

    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream(dev)
    cases = [(19, 5, 94), (11, 64, 95)]
    Js = [W.random_instances(N, I, seed) for N, I, seed in cases]
    wants = [pkg.ground_energy(N, J) for (N, _, _), J in zip(cases, Js)]
    J_devs = [torch.from_numpy(J).to(dev) for J in Js]
    e_devs = [torch.full((I,), -7, dtype=torch.int64, device=dev) for _, I, _ in cases]
    torch.cuda.synchronize()
    for (N, I, _), J_dev, e_dev in zip(cases, J_devs, e_devs):
        assert _call(N, I, J_dev, e_dev, s.cuda_stream) == pkg.SQA_OK, pkg.lib().sqa_last_error()
    s.synchronize()
    for k, (e_dev, want) in enumerate(zip(e_devs, wants)):
        assert np.array_equal(e_dev.cpu().numpy(), want), f"queued call {k}"
    # the binding's wrapper gives the same
    e2 = torch.zeros_like(e_devs[0])
    with torch.cuda.stream(s):
        pkg.ground_energy_noalloc(cases[0][0], J_devs[0], e2, stream=s)
    s.synchronize()
    assert np.array_equal(e2.cpu().numpy(), wants[0])


def test_noalloc_rejects_sizes_beyond_its_scratch_and_budget():
    import torch

    dev = torch.device("cuda", 0)
    J_dev = torch.zeros((1, 1), dtype=torch.int32, device=dev)
    e_dev = torch.zeros((1,), dtype=torch.int64, device=dev)
    st = pkg.lib().sqa_ground_energy_noalloc(2, 4097, J_dev.data_ptr(), e_dev.data_ptr(), None)
    assert st == pkg.SQA_ERR_INVALID
    assert b"4096" in pkg.lib().sqa_last_error()
    # more than 2^40 states in all: refused before any launch
    st = pkg.lib().sqa_ground_energy_noalloc(40, 3, J_dev.data_ptr(), e_dev.data_ptr(), None)
    assert st == pkg.SQA_ERR_UNSUPPORTED
    assert b"budget" in pkg.lib().sqa_last_error()


def test_noalloc_rejects_host_buffers_and_bad_tensors():
    import torch

    dev = torch.device("cuda", 0)
    J = W.random_instances(6, 2, 96)
    e = np.zeros(2, np.int64)
    # host memory is refused by the pointer check, before any launch
    st = pkg.lib().sqa_ground_energy_noalloc(6, 2, J.ctypes.data, e.ctypes.data, None)
    assert st == pkg.SQA_ERR_INVALID
    J_dev = torch.from_numpy(J).to(dev)
    with pytest.raises(ValueError):
        pkg.ground_energy_noalloc(6, J_dev.to(torch.int64), torch.zeros(2, dtype=torch.int64, device=dev))
    with pytest.raises(ValueError):
        pkg.ground_energy_noalloc(6, J_dev[:, :10].contiguous(), torch.zeros(2, dtype=torch.int64, device=dev))
    with pytest.raises(ValueError):
        pkg.ground_energy_noalloc(6, J_dev, torch.zeros(3, dtype=torch.int64, device=dev))
