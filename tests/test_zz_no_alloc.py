"""dtw_align_static: the allocation-free entry point, checked against dtw_align.

Callers that cannot allocate device memory while they align (a real-time
loop that must not block in the driver's allocator, or a process whose device
memory is already reserved by another allocator) use dtw_align_static, which
keeps all of its scratch in one fixed device array.  This file is collected
last on purpose (test_zz_*): if it fails, a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2607_15478_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2607_15478_gb300 import build, pardtw
    build.build()
    pardtw.load_library()
    return pardtw


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def run_static(pardtw, A, B):
    cap = min(A.shape[0], B.shape[0])
    path = torch.full((cap, 2), -7, dtype=torch.int32, device="cuda")
    plen = torch.zeros(1, dtype=torch.int32, device="cuda")
    tot = torch.zeros(1, dtype=torch.float32, device="cuda")
    pardtw.dtw_align_static(A, B, path, plen, tot)
    n = int(plen.item())  # synchronises the current stream
    assert n > 0, pardtw.status_string(-n) if n < 0 else "empty path"
    return path[:n].cpu().numpy(), float(tot.item())


def test_static_matches_dtw_align_on_two_calls_in_a_row(lib):
    pardtw = lib
    cases = [synth.config_pair(0),                         # 1000 x 1200
             synth.config_pair(1, La=3000, Lb=3600)]       # larger, then reuse the scratch
    with pardtw.Aligner(0) as al:
        for wp in cases:
            A, B = dev(wp.A), dev(wp.B)
            p_ref, t_ref = al.align(A, B)
            p_st, t_st = run_static(pardtw, A, B)
            # the same DP cells (the transposed sweep dtw_align may take gives
            # bit-identical cells) and the same end cell: path and total equal
            # bit for bit
            np.testing.assert_array_equal(p_st, p_ref.cpu().numpy())
            assert t_st == t_ref


def test_static_timeout_then_recovers(lib):
    # a bounded device wait that expires (the first strip group never
    # publishes its border; the wait gives up after 20 ms) is reported through
    # path_len = -DTW_ERR_TIMEOUT; the next call on the same array, which
    # still holds that call's state, aligns correctly
    pardtw = lib
    wp = synth.config_pair(0)
    A, B = dev(wp.A), dev(wp.B)
    path = torch.zeros((1000, 2), dtype=torch.int32, device="cuda")
    plen = torch.zeros(1, dtype=torch.int32, device="cuda")
    opt = pardtw.make_options(wait_limit_us=20000, debug_skip_publish=0)
    pardtw.dtw_align_static(A, B, path, plen, options=opt)
    assert int(plen.item()) == -pardtw.DTW_ERR_TIMEOUT
    with pardtw.Aligner(0) as al:
        p_ref, t_ref = al.align(A, B)
    p_st, t_st = run_static(pardtw, A, B)
    np.testing.assert_array_equal(p_st, p_ref.cpu().numpy())
    assert t_st == t_ref


def test_static_rejects_host_buffers(lib):
    # staging a host buffer would need scratch of its own: host pointers are
    # refused before any work is queued
    pardtw = lib
    wp = synth.config_pair(0, La=200, Lb=240)
    path = torch.zeros((200, 2), dtype=torch.int32, device="cuda")
    plen = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pardtw.PardtwError) as e:
        pardtw.dtw_align_static(torch.from_numpy(wp.A), dev(wp.B), path, plen)
    assert e.value.status == pardtw.DTW_ERR_INVALID
    with pytest.raises(pardtw.PardtwError) as e:
        pardtw.dtw_align_static(dev(wp.A), dev(wp.B), path, torch.zeros(1, dtype=torch.int32))
    assert e.value.status == pardtw.DTW_ERR_INVALID


def test_static_rejects_sizes_beyond_its_scratch(lib):
    pardtw = lib
    assert pardtw.dtw_static_scratch_bytes() == 64 << 20
    A = torch.zeros((20000, 12), dtype=torch.float32, device="cuda")
    B = torch.zeros((25000, 12), dtype=torch.float32, device="cuda")
    path = torch.zeros((20000, 2), dtype=torch.int32, device="cuda")
    plen = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pardtw.PardtwError) as e:
        pardtw.dtw_align_static(A, B, path, plen)
    assert e.value.status == pardtw.DTW_ERR_SCRATCH_LIMIT
