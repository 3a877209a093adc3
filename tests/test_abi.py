"""The C-ABI library builds, loads without a GPU and exports what include/*.h declares."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2607_15478_gb300 import build as pbuild
from paper_2607_15478_gb300 import pardtw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(?:int|void|size_t|const char\s*\*)\s+(dtw_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return pardtw.load_library()


def test_header_declares_the_binding_exports():
    assert declared_functions() == set(pardtw.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for s in range(7):
        assert pardtw.status_string(s)
    assert "unreachable" in pardtw.status_string(pardtw.DTW_ERR_UNREACHABLE)


def test_default_options(lib):
    o = pardtw.make_options()
    assert o.cost_precision == pardtw.DTW_COST_FP32
    assert o.cost_shift == 0.0 and o.debug_skip_publish == -1


def _layout_bytes(rows, cols, rps, words, spg):
    """The dominant buffers of one sweep orientation: 2-bit fields (words per
    strip and 16-column chunk), tagged border rows (16 B per column and
    group of spg strips), band maps of the parallel backtrace (8 B per column
    per 128-row band, again for every other band and for every fourth)."""
    nstrips = -(-rows // rps)
    bp = nstrips * words * -(-cols // 16) * 4
    border = -(-nstrips // spg) * cols * 16
    nbands = -(-rows // 128)
    n2 = (nbands - 2) // 2 if nbands >= 4 else 0
    n4 = (nbands - 6) // 4 + 1 if nbands >= 6 else 0
    maps = (nbands + n2 + n4) * cols * 8
    return bp + border + maps


def test_workspace_size_follows_memory_model(lib):
    # Sec. VI-D: the 2-bit backtrace matrix (L^2 / 4 bytes) plus O(L)
    # buffers; here also the tagged border rows between strip groups and the
    # band entry maps of the parallel backtrace.  Default options: 3 rows per
    # lane (93-row strips, 96 words), two strips per CTA; either orientation
    # of the sweep.
    for La, Lb in [(1000, 1200), (20000, 25000), (100000, 130000)]:
        n = pardtw.workspace_size(La, Lb, 12)
        extra = max(_layout_bytes(La, Lb, 93, 96, 2), _layout_bytes(Lb, La, 93, 96, 2))
        assert extra <= n <= extra * 1.01 + 64 * (La + Lb) * 12
        # about 0.46 bytes per cell
        if La >= 20000:
            assert 0.45 <= n / (La * Lb) <= 0.47
    # one row per lane (30-row strips of 32 words, four strips per CTA)
    n1 = pardtw.workspace_size(20000, 25000, 12, pardtw.make_options(rows_per_lane=1))
    extra = max(_layout_bytes(20000, 25000, 30, 32, 4), _layout_bytes(25000, 20000, 30, 32, 4))
    assert extra <= n1 <= extra * 1.01 + 64 * 45000 * 12
    with pytest.raises(pardtw.PardtwError):
        pardtw.workspace_size(0, 10, 12)


def test_largest_square_pair_on_gb300(lib):
    # Sec. VI-D sizes the longest pair by the memory the 2-bit matrix takes:
    # L_max = 2^16 sqrt(T) for T GB (1.10e6 frames for the 280 GB of a GB300
    # that a process can use).  With the border rows and band maps this
    # library needs 0.46 bytes per cell: the largest square pair is ~0.78e6
    # frames (0.72 of the paper's bound), found here by bisection on
    # dtw_workspace_size.
    budget = 280e9
    lo, hi = 1000, 2_000_000
    while hi - lo > 1000:
        mid = (lo + hi) // 2
        if pardtw.workspace_size(mid, mid, 12) <= budget:
            lo = mid
        else:
            hi = mid
    paper = 2 ** 16 * (280.0 ** 0.5)
    assert 775_000 <= lo <= 795_000, lo
    assert 0.70 <= lo / paper <= 0.73
    assert pardtw.workspace_size(lo, lo, 12) <= budget < pardtw.workspace_size(lo + 1000, lo + 1000, 12)


def test_workspace_size_rejects_unsupported_dim(lib):
    with pytest.raises(pardtw.PardtwError) as e:
        pardtw.workspace_size(10, 10, 4096)
    assert e.value.status == pardtw.DTW_ERR_UNSUPPORTED


def test_create_without_gpu_fails_cleanly(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    h = ctypes.c_void_p()
    rc = lib.dtw_create(ctypes.byref(h), 0, None)
    assert rc in (pardtw.DTW_ERR_CUDA, pardtw.DTW_ERR_INVALID)
    assert h.value is None


def test_encoder_parameter_count_matches_layout(lib):
    # the flat parameter array of the learned band's encoder (include/pardtw.h)
    from paper_2607_15478_gb300 import band_train
    for D in (1, 12, 32, 64):
        lay, n = band_train.layout(D)
        assert pardtw.dtw_encoder_param_count(D) == n
        assert n == 64 * D * 5 + 64 + 2 * (64 * 64 * 5 + 64) + 16 * 64 + 16 + 64 + 1
    assert pardtw.dtw_encoder_param_count(0) == 0
    assert pardtw.dtw_encoder_param_count(65) == 0


def test_encoder_init_params():
    from paper_2607_15478_gb300 import band_train
    p = band_train.init_params(12, seed=0)
    lay, n = band_train.layout(12)
    assert p.shape == (n,) and p.dtype.name == "float32"
    o, shp = lay["W2"]
    w2 = p[o:o + 64 * 64 * 5]
    lim = (6.0 / (64 * 5)) ** 0.5
    assert np.abs(w2).max() <= lim and abs(w2.std() - lim / 3 ** 0.5) < 0.05 * lim
    assert p[lay["b5"][0]] == -2.0
    assert np.array_equal(p, band_train.init_params(12, seed=0))
