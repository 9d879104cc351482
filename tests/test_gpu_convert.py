"""The library's FP32 <-> FP64 conversion kernel (chebmg_convert), which the mixed-precision solve
uses between its FP64 Krylov vectors and its FP32 V-cycle and which converts in integer
arithmetic: it must give the hardware's IEEE result bit for bit.  Widening is checked on every
one of the 2^32 float bit patterns; narrowing on every double exponent that maps into or next to
the float range, with random mantissas and every rounding case (below, at and above the halfway
point of the 29 dropped bits, with an even and an odd last kept bit), and on the special values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2210_03179_gb300 as cm  # noqa: E402


def _same_bits_or_both_nan(got, ref):
    got_nan, ref_nan = torch.isnan(got), torch.isnan(ref)
    assert torch.equal(got_nan, ref_nan)
    ib = torch.int64 if got.dtype == torch.float64 else torch.int32
    keep = ~ref_nan
    assert torch.equal(got.view(ib)[keep], ref.view(ib)[keep])


def test_widening_every_float_bit_pattern():
    chunk = 1 << 28
    for start in range(0, 1 << 32, chunk):
        bits = torch.arange(start, start + chunk, dtype=torch.int64, device="cuda")
        bits = torch.where(bits >= (1 << 31), bits - (1 << 32), bits).to(torch.int32)
        x = bits.view(torch.float32)
        y = torch.empty(chunk, dtype=torch.float64, device="cuda")
        cm.chebmg_convert(x, y)
        _same_bits_or_both_nan(y, x.to(torch.float64))
        del bits, x, y


def _doubles_for_narrowing():
    rng = np.random.default_rng(5)
    out = []
    tie = 1 << 28
    for e in range(880, 1170):                    # float exponents -16 .. 273 (subnormal to overflow)
        m = rng.integers(0, 1 << 52, 2048, dtype=np.uint64)
        low = m & np.uint64((1 << 29) - 1)
        hi = m & ~np.uint64((1 << 29) - 1)
        cases = [m]
        for r in (0, 1, tie - 1, tie, tie + 1, (1 << 29) - 1):
            for lsb in (0, 1):                    # even and odd last kept bit
                cases.append((hi & ~np.uint64(1 << 29)) | np.uint64(lsb << 29) | np.uint64(r))
        for c in cases:
            for sign in (0, 1):
                out.append((np.uint64(sign) << np.uint64(63)) | (np.uint64(e) << np.uint64(52)) | c)
        del low
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028234663852886e38, 3.4028235677973366e38,
                        -3.4028235677973366e38, 1.1754943508222875e-38, 1.1754942106924411e-38, 1e-45, 1e300],
                       dtype=np.float64).view(np.uint64)
    out.append(special)
    return np.concatenate(out).view(np.float64)


def test_narrowing_matches_ieee_round_to_nearest_even():
    x = torch.tensor(_doubles_for_narrowing(), device="cuda")
    y = torch.empty(x.numel(), dtype=torch.float32, device="cuda")
    cm.chebmg_convert(x, y)
    _same_bits_or_both_nan(y, x.to(torch.float32))


def test_same_precision_copies_and_bad_arguments():
    x = torch.randn(1001, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    cm.chebmg_convert(x, y)
    assert torch.equal(x, y)
    with pytest.raises(ValueError):
        cm.chebmg_convert(x, torch.empty(5, dtype=torch.float32, device="cuda"))
