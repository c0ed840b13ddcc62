"""The integer-only FP64/FP32 conversions of the kernels (hfd_check_conversions) equal the
hardware conversions bit for bit: round to nearest even from FP64 to FP32 over the whole float
range (ties, subnormal results, overflow to infinity), and exact widening of every class of
float (subnormals, zeros, infinities)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(seed=11):
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    # random significands over exponents from far below the float range to above it
    e = rng.integers(-170, 140, 400000)
    parts.append(rng.uniform(1.0, 2.0, e.size) * np.ldexp(1.0, e) * rng.choice([-1.0, 1.0], e.size))
    # exact ties and near-ties between neighbouring floats, normal and subnormal
    f = np.concatenate([rng.uniform(-3e4, 3e4, 50000),
                        np.ldexp(rng.uniform(1.0, 2.0, 50000), rng.integers(-149, -126, 50000)),
                        np.ldexp(rng.uniform(1.0, 2.0, 50000), rng.integers(-126, 127, 50000))])
    f32 = f.astype(np.float32)
    nxt = np.nextafter(f32, np.float32(np.inf)).astype(np.float64)
    mid = 0.5 * (f32.astype(np.float64) + nxt)
    parts += [mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf)]
    # edges of the range and special values
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).smallest_subnormal)
    parts.append(np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, 2.0 ** 128,
                           fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -24), tiny, 0.5 * tiny,
                           0.75 * tiny, 0.5 * tiny * (1 + 2.0 ** -40), 2.0 ** -126,
                           2.0 ** -126 * (1 - 2.0 ** -25), 1e-300, -1e-310, 5e-324, 1.0, -1.0]))
    # low 32 bits as float patterns: random words plus every exponent class
    words = rng.integers(0, 2 ** 32, 200000, dtype=np.uint64)
    special = np.array([0, 0x80000000, 1, 0x807fffff, 0x007fffff, 0x00800000, 0x7f7fffff,
                        0x7f800000, 0xff800000, 0x7fc00000, 0x3f800000], dtype=np.uint64)
    hi = rng.integers(0, 2 ** 32, words.size + special.size, dtype=np.uint64) << np.uint64(32)
    patt = (hi | np.concatenate([words, special])).view(np.float64)
    parts.append(patt)
    return np.concatenate(parts)


def test_integer_conversions_equal_hardware_conversions():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_01286_gb300.hfd import check_conversions
    x = torch.from_numpy(_inputs()).cuda()
    f_int, f_hw, d_int, d_hw = (t.cpu() for t in check_conversions(x))
    nan_f = torch.isnan(f_hw)
    assert torch.equal(torch.isnan(f_int), nan_f)
    assert torch.equal(f_int.view(torch.int32)[~nan_f], f_hw.view(torch.int32)[~nan_f])
    nan_d = torch.isnan(d_hw)
    assert torch.equal(torch.isnan(d_int), nan_d)
    assert torch.equal(d_int.view(torch.int64)[~nan_d], d_hw.view(torch.int64)[~nan_d])
    # the inputs reach every class: subnormal and infinite results, both tie directions
    fb = f_hw[~nan_f]
    assert (fb.abs() < float(np.finfo(np.float32).tiny)).logical_and(fb != 0).any()
    assert torch.isinf(fb).sum() > 3
    # and the host's conversion (numpy) agrees with the device's on the finite inputs
    xn = x.cpu().numpy()
    with np.errstate(over="ignore", invalid="ignore"):
        ref = xn.astype(np.float32)
    fin = ~np.isnan(xn)
    assert np.array_equal(f_hw.numpy()[fin].view(np.int32), ref[fin].view(np.int32))


def test_conversion_check_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_01286_gb300.hfd import check_conversions
    with pytest.raises(TypeError):
        check_conversions(torch.zeros(4, dtype=torch.float32, device="cuda"))
    out = check_conversions(torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert all(t.numel() == 0 for t in out)
