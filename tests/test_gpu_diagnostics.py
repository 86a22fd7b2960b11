"""The integer-pipe probe behind the bench's ALU rooflines: every op gives a
positive rate, an unknown op is refused, and the outer-product form of the
batched kernel (both factors in registers) runs no faster than the fused
constant-factor form."""
import ctypes
import math

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2003_12197_gb300 as H  # noqa: E402


def test_int_pipe_rates():
    H.build_library()
    r = H.hers_probe_int_pipe(0, iters=1 << 12)
    assert set(r) == set(H.INT_PIPE_OPS)
    for name, v in r.items():
        assert math.isfinite(v) and v > 1e11, (name, v)
    # one SM-wide IMAD.WIDE per 4 cycles per sub-partition bounds both forms
    assert r["mad_wide_s32_outer"] < 1.2 * r["imad_wide_u32"]


def test_int_pipe_unknown_op_is_refused():
    H.build_library()
    v = ctypes.c_double()
    assert H.lib().hers_probe_int_pipe(0, len(H.INT_PIPE_OPS), 1024, ctypes.byref(v)) == -1  # HERS_E_INVAL
    assert H.lib().hers_probe_int_pipe(0, 0, 0, ctypes.byref(v)) == -1  # HERS_E_INVAL
