"""The FP32-form kernels convert between FP64 and FP32 with integer field
moves (the hardware conversion issues on the FP64 pipe).  Checked bit for bit
against the hardware conversions (torch's .to on the GPU) over random values
of every magnitude, round-to-nearest-even ties on both sides, the edges of
the float range, subnormals, signed zeros, infinities and NaN."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csl():
    import __graft_entry__ as g
    g.build()
    import paper_2408_00488_gb300 as csl
    return csl


def doubles():
    rng = np.random.default_rng(41)
    # random sign, mantissa and exponent over the whole float range and beyond
    m = rng.uniform(1.0, 2.0, 200000)
    e = rng.integers(-160, 140, 200000)
    x = np.ldexp(m, e) * rng.choice([-1.0, 1.0], 200000)
    # exact ties: a float mantissa plus exactly half an ulp (odd and even kept parts)
    f = rng.uniform(-1e30, 1e30, 50000).astype(np.float32)
    up = np.nextafter(f, np.float32(np.inf))
    ties = (f.astype(np.float64) + up.astype(np.float64)) / 2
    near = [np.float64(3.4028234663852886e38), np.float64(3.4028235677973366e38), np.float64(3.4028236e38),
            np.float64(1.1754943508222875e-38), np.float64(1.1754942e-38), np.float64(1e-40), np.float64(1e-46),
            0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 0.1, 1.0 / 3.0]
    return np.concatenate([x, ties, np.array(near, dtype=np.float64)])


def test_d2f_matches_hardware_round_to_nearest(csl):
    import torch
    x = torch.from_numpy(doubles()).cuda()
    ours = csl._binding.test_convert(x, torch.float32)
    hw = x.to(torch.float32)
    a, b = ours.cpu().numpy(), hw.cpu().numpy()
    nan = np.isnan(b)
    assert np.array_equal(np.isnan(a), nan)
    assert np.array_equal(a[~nan].view(np.uint32), b[~nan].view(np.uint32))


def test_f2d_is_exact(csl):
    import torch
    rng = np.random.default_rng(42)
    bits = rng.integers(0, 2**32, 300000, dtype=np.uint64).astype(np.uint32)
    f = np.concatenate([bits.view(np.float32),
                        np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.17549435e-38,
                                  3.4028235e38], dtype=np.float32)])
    x = torch.from_numpy(f).cuda()
    ours = csl._binding.test_convert(x, torch.float64)
    hw = x.to(torch.float64)
    a, b = ours.cpu().numpy(), hw.cpu().numpy()
    nan = np.isnan(b)
    assert np.array_equal(np.isnan(a), nan)
    assert np.array_equal(a[~nan].view(np.uint64), b[~nan].view(np.uint64))
