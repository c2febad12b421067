"""The hand-written elementary functions of the rollout and repair kernels,
evaluated on the GPU through smppi_debug_elementary on dense grids of their
domains, against float64 (numpy) and against CUDA's own functions of the same
float32 arguments.  Errors are in ulps of the float32 result.

  * atan2 (octant reduction + the minimax polynomial), scalar and packed form
    (Horner, and the one-thread recurrences' Estrin form with the octant folded
    into one FMA), for finite arguments with max(|x|, |y|) in [2^-126, 2^126) and at the
    special points (0, 0), (+-0, x), (y, 0): within 4 ulp (3.8 measured: up to
    3 from the reciprocal and the polynomial, 0.7 from the float32 pi/2 of the
    octant fold);
  * sin(1.5 atan z) by the half-angle identities (the C = 1.5 tyre), scalar
    and packed: within 6 ulp (5.0 measured: two reciprocal square roots and
    three products), and where the result is below 1e-30 in size within 1e-36
    absolutely;
  * sin and cos of |x| <= 1/2 by the Taylor series (scalar to x^9 / x^10,
    packed to x^7 / x^8): within 2 ulp.
The maxima are printed next to those of CUDA's atan2f / sinf(1.5 atanf) /
sinf / cosf on the same arguments.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_11719_gb300 import smppi
    return smppi


def _run(S, fn, a, b=None):
    a = np.ascontiguousarray(a, np.float32)
    b = np.zeros_like(a) if b is None else np.ascontiguousarray(b, np.float32)
    ad, bd = torch.as_tensor(a, device="cuda"), torch.as_tensor(b, device="cuda")
    out, ref = torch.empty_like(ad), torch.empty_like(ad)
    S.smppi_debug_elementary(fn, ad, bd, out, ref)
    torch.cuda.synchronize()
    return a, b, out.cpu().numpy(), ref.cpu().numpy()


def _ulp(v64):
    r = np.abs(v64).astype(np.float32)
    return np.maximum(np.spacing(r).astype(np.float64), float(np.spacing(np.float32(1.17549435e-38))))


def _ulp_err(out, exact):
    return np.abs(out.astype(np.float64) - exact) / _ulp(exact)


def _atan2_args(rng):
    th = np.linspace(-np.pi, np.pi, 200001)
    ys, xs = [], []
    for r in (1e-30, 1e-3, 0.7, 1.0, 3.0, 1e3, 1e30):
        ys.append(r * np.sin(th))
        xs.append(r * np.cos(th))
    n = 200000
    mag = lambda: np.exp(rng.uniform(np.log(1.2e-38 * 8), np.log(8e37), n))   # noqa: E731
    ys.append(mag() * rng.choice([-1.0, 1.0], n))
    xs.append(mag() * rng.choice([-1.0, 1.0], n))
    # slip-angle-like arguments: (v_y + l r, v_x) with |v_x| of a few m/s
    ys.append(rng.normal(0, 3, n))
    xs.append(rng.uniform(-10, 10, n))
    special_y = [0.0, -0.0, 0.0, -0.0, 1.0, -1.0, 5.0, -5.0, 1e-20, -1e-20]
    special_x = [0.0, 0.0, 2.0, 2.0, 0.0, 0.0, -0.0, 0.0, -3.0, -3.0]
    ys.append(np.array(special_y))
    xs.append(np.array(special_x))
    return np.concatenate(ys).astype(np.float32), np.concatenate(xs).astype(np.float32)


@pytest.mark.parametrize("fn,name", [(0, "scalar"), (1, "packed"), (8, "packed, Estrin + folded octant")])
def test_atan2(S, fn, name):
    y, x, out, ref = _run(S, fn, *_atan2_args(np.random.default_rng(1)))
    exact = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    e = _ulp_err(out, exact)
    e_cuda = _ulp_err(ref, exact)
    print("atan2 (%s), %d arguments: max %.2f ulp (CUDA atan2f %.2f ulp)"
          % (name, y.size, e.max(), e_cuda.max()))
    assert e.max() <= 4.0
    # the special points exactly, signs included
    assert out[-10] == 0.0 and out[-8] == 0.0 and np.signbit(out[-7])
    assert out[-6] == np.float32(np.pi / 2) or abs(out[-6] - np.pi / 2) <= 2.4e-7


@pytest.mark.parametrize("fn,name", [(2, "scalar"), (3, "packed")])
def test_tyre_half_angle(S, fn, name):
    z = np.concatenate([np.sinh(np.linspace(-12.0, 12.0, 400001)), [0.0, -0.0, 1e-30, -1e-30,
                                                                      1e18, -1e18]])
    z, _, out, ref = _run(S, fn, z)
    exact = np.sin(1.5 * np.arctan(z.astype(np.float64)))
    e = _ulp_err(out, exact)
    e_cuda = _ulp_err(ref, exact)
    tiny = np.abs(exact) < 1e-30
    print("sin(1.5 atan z) (%s), %d arguments: max %.2f ulp (CUDA sinf(1.5f atanf) %.2f ulp)"
          % (name, z.size, e[~tiny].max(), e_cuda[~tiny].max()))
    assert e[~tiny].max() <= 6.0
    assert np.all(np.abs(out[tiny] - exact[tiny]) <= 1e-36)


@pytest.mark.parametrize("fn_s,fn_c,name", [(4, 5, "scalar"), (6, 7, "packed")])
def test_sincos_half(S, fn_s, fn_c, name):
    x = np.concatenate([np.linspace(-0.5, 0.5, 1000001), [0.0, -0.0, 1e-30, -1e-30]])
    x, _, s_out, s_ref = _run(S, fn_s, x)
    _, _, c_out, c_ref = _run(S, fn_c, x)
    x64 = x.astype(np.float64)
    es, ec = _ulp_err(s_out, np.sin(x64)), _ulp_err(c_out, np.cos(x64))
    print("sin / cos on [-1/2, 1/2] (%s): max %.2f / %.2f ulp (CUDA sinf / cosf %.2f / %.2f ulp)"
          % (name, es.max(), ec.max(), _ulp_err(s_ref, np.sin(x64)).max(),
             _ulp_err(c_ref, np.cos(x64)).max()))
    assert es.max() <= 2.0 and ec.max() <= 2.0


def test_rsqrt_without_denormal_path_is_rsqrtf(S):
    """The tyre and Box-Muller take 1/sqrt of arguments that are never denormal
    (1 + z^2, (1 + cos t)/2, -2 ln u >= 1.2e-7) by rsqrt.approx.ftz: bit for bit
    rsqrtf on every float in [1/2, 2) (both mantissa phases of the square root)
    and on samples of every normal binade, with the special values."""
    grid = np.arange(np.float32(0.5).view(np.uint32), np.float32(2.0).view(np.uint32),
                     dtype=np.uint32).view(np.float32)
    rng = np.random.default_rng(5)
    bits = (rng.integers(1, 254, 2000000, dtype=np.uint32) << 23) | \
        rng.integers(0, 1 << 23, 2000000, dtype=np.uint32)
    x = np.concatenate([grid, bits.view(np.float32),
                        np.array([np.inf, 1.17549435e-38, 3.4028235e38], np.float32)])
    _, _, out, ref = _run(S, 9, x)
    same = out.view(np.uint32) == ref.view(np.uint32)
    print("rsqrt without denormal path: %d of %d arguments bit-equal to rsqrtf"
          % (int(same.sum()), x.size))
    assert np.all(same)

