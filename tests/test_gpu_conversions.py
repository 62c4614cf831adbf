"""The integer-pipe FP32 <-> FP64 conversions of the batched kernels (written from the IEEE-754
binary32 / binary64 layouts) against the hardware conversions, bit for bit, over hashed bit
patterns of every class, doubles near the float range and rounding ties."""
import ctypes

import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [1, 0x5eed, 2 ** 63 + 7])
def test_integer_conversions_match_hardware(seed):
    torch = need_gpu()
    from paper_2306_02526_gb300 import _lib
    bad = ctypes.c_int64(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = _lib.lib().hps_selftest_conversions(1 << 22, seed, stream, ctypes.byref(bad))
    assert rc == _lib.HPS_OK
    assert bad.value == 0
