"""The mixed path's five-digit split, emulated exactly in numpy, against the bounds its design
relies on (the tensor-core contraction of eq 9 on 8-bit digits):

* every stored digit is an integer of at most 8 significant bits (exact in BF16), |s_k| <= 128
  except s2 <= 130 where the lo word joins after digit 1 (unnormalised products);
* the five digits reconstruct each value to 2^-38 of its window's largest: the last digit's
  rounding leaves 2^-33 of the scaled unit and the lo word's join rounds once more at most as
  much, against a largest scaled value of at least 64 (the digits span 39 bits);
* the order-k sums sum_{i+j=k} s_i t_j over a 128-point window stay below 2^24 in digit units,
  so FP32 accumulation of the slice products is exact;
* the fold (order 1 split at 2^24, one TwoSum into the double-float sum, orders 2-4 as one
  FP32 term) accumulates windows to within 2^-38 of sum_w 128 max|a_w| max|b_w| of the exact
  dot product of the double-float inputs.

Each kernel step is an FP32 add or FMA whose exact result fits in an FP64 significand (a power
-of-two scale times an FP32 value plus a multiple of the spacing), so computing it in FP64 and
rounding once to FP32 gives the correctly rounded FP32 result.  The emulation follows the
steps: t = v sc + 1.5 2^23 (digit 0 rounds inside its FMA), stored digit fma(t, -256,
1.5 2^31) = -256 s, remainder fma(r, 256, -256 s); lo joins after digit JOIN."""
import numpy as np

M = np.float32(1.5 * 2.0 ** 23)
M256 = 1.5 * 2.0 ** 31


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def split(vh, vl, e, join=1, n=5):
    """Stored digits (-256 s_k, FP32) of the double-float values (vh, vl) of one window whose
    largest |value| is below 2^e."""
    sc = 2.0 ** (7 - e)
    scj = 2.0 ** (7 - e + 8 * (join + 1))
    lo = f32(vl.astype(np.float64) * scj)
    digits = []
    r = None
    for k in range(n):
        t = f32(vh.astype(np.float64) * sc + float(M)) if k == 0 else f32(r.astype(np.float64) + float(M))
        d = f32(t.astype(np.float64) * -256.0 + M256)
        digits.append(d)
        if k + 1 < n:
            if k == 0:
                r = f32(vh.astype(np.float64) * (sc * 256.0) + d.astype(np.float64))
            else:
                r = f32(r.astype(np.float64) * 256.0 + d.astype(np.float64))
            if k == join:
                r = f32(r.astype(np.float64) + lo.astype(np.float64))
    return np.stack(digits)


def unnormalised_products(rng, n, span):
    """Double-float products left unnormalised, as the kernels form them: hi = fl(xh yh),
    lo = the product's rounding error plus the cross terms (|lo| <= 3 2^-24 |hi|)."""
    x = rng.standard_normal(n) * np.exp(rng.uniform(-span, 0, n))
    y = rng.standard_normal(n) * np.exp(rng.uniform(-span, 0, n))
    xh, yh = f32(x), f32(y)
    xl, yl = f32(x - xh.astype(np.float64)), f32(y - yh.astype(np.float64))
    h = f32(xh.astype(np.float64) * yh)
    err = xh.astype(np.float64) * yh - h.astype(np.float64)  # exact in FP64
    lo = f32(f32(err + xh.astype(np.float64) * yl) + xl.astype(np.float64) * yh)
    return h, lo, h.astype(np.float64) + lo.astype(np.float64)


def window_exponent(vh):
    mx = float(np.max(np.abs(vh)))
    return int(np.frexp(mx)[1])  # mx < 2^e <= 2 mx


def test_digits_are_bf16_exact_and_bounded():
    rng = np.random.default_rng(5)
    worst = np.zeros(5)
    for span in (0.0, 3.0, 12.0, 40.0):
        for _ in range(40):
            vh, vl, _ = unnormalised_products(rng, 128, span)
            d = split(vh, vl, window_exponent(vh))
            s = -d.astype(np.float64) / 256.0
            assert np.all(s == np.round(s))
            bits = d.view(np.uint32)
            assert np.all(bits & 0xFFFF == 0)  # the low 16 bits are zero: exact in BF16
            worst = np.maximum(worst, np.abs(s).max(axis=1))
    assert worst[0] <= 128 and worst[1] <= 128 and worst[3] <= 128 and worst[4] <= 128, worst
    assert worst[2] <= 130, worst


def test_five_digits_reconstruct_to_2_38_of_the_window():
    rng = np.random.default_rng(6)
    worst = 0.0
    for span in (0.0, 5.0, 20.0):
        for _ in range(40):
            vh, vl, v = unnormalised_products(rng, 128, span)
            e = window_exponent(vh)
            s = -split(vh, vl, e).astype(np.float64) / 256.0
            back = sum(s[k] * 256.0 ** -k for k in range(5)) * 2.0 ** (e - 7)
            err = np.abs(back - v).max() / np.abs(v).max()
            assert err <= 2.0 ** -38, (span, err)
            worst = max(worst, err)
    assert worst > 2.0 ** -40  # the bound is reached to within a small factor


def test_order_sums_are_exact_in_fp32():
    """Worst order-k sums over 128 points of random windows, with every digit product taken at
    its absolute value (all terms of one sign), against the design's bound."""
    rng = np.random.default_rng(7)
    top = 0.0
    for _ in range(60):
        ah, al, _ = unnormalised_products(rng, 128, 1.0)
        bh, bl, _ = unnormalised_products(rng, 128, 1.0)
        sa = np.abs(split(ah, al, window_exponent(ah)).astype(np.float64) / 256.0)
        sb = np.abs(split(bh, bl, window_exponent(bh)).astype(np.float64) / 256.0)
        for k in range(5):
            tot = sum(float(np.sum(sa[i] * sb[k - i])) for i in range(k + 1))
            top = max(top, tot)
    bound = 128 * 114688  # the design's bound: 128 points x 7 x 128^2
    assert top < bound < 2 ** 24, (top, bound)


def _two_sum(a, b):
    s = np.float32(a + b)
    bb = np.float32(s - a)
    return s, np.float32(np.float32(a - np.float32(s - bb)) + np.float32(b - bb))


def _fast_two_sum(a, b):
    s = np.float32(a + b)
    return s, np.float32(b - np.float32(s - a))


def _fma(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _fold(o, sc, H, L):
    """One window's five order sums into the running double-float sum (H, L), step by step as
    the fold warps do it."""
    mag = np.float32(1.5 * 2.0 ** 47)
    q1 = np.float32(np.float32(o[1] + mag) - mag)  # nearest multiple of 2^24
    r1 = np.float32(o[1] - q1)
    s0h, s0l = _two_sum(H, np.float32(_fma(q1, np.float32(2.0 ** -8), o[0]) * sc))
    tail = np.float32(_fma(r1, np.float32(2.0 ** -8), _fma(o[2], np.float32(2.0 ** -16), _fma(
        o[4], np.float32(2.0 ** -32), np.float32(o[3] * np.float32(2.0 ** -24))))) * sc)
    lo = np.float32(L + np.float32(s0l + tail))
    return _fast_two_sum(s0h, lo)


def test_window_fold_matches_the_exact_dot_product():
    """Digits of one A row and one B column per window, their exact order sums (as the tensor
    cores accumulate them), the fold with the window scales 2^(e_a - 15) 2^(e_b - 15): against
    the exact sum of the double-float products over 1-19 windows (measured worst 2^-41.3 of
    the window bound)."""
    import math
    rng = np.random.default_rng(8)
    worst = 0.0
    for _ in range(120):
        span = float(rng.choice([0.0, 3.0, 10.0]))
        H = L = np.float32(0.0)
        exact = bound = 0.0
        for _w in range(int(rng.integers(1, 20))):
            ah, al, a = unnormalised_products(rng, 128, span)
            bh, bl, b = unnormalised_products(rng, 128, span)
            ea, eb = window_exponent(ah), window_exponent(bh)
            da = split(ah, al, ea).astype(np.float64)
            db = split(bh, bl, eb).astype(np.float64)
            o = []
            for k in range(5):
                ok = sum(float(np.dot(da[i], db[k - i])) for i in range(k + 1))
                assert float(np.float32(ok)) == ok  # exact in FP32
                o.append(np.float32(ok))
            H, L = _fold(o, np.float32(2.0 ** (ea - 15) * 2.0 ** (eb - 15)), H, L)
            exact += math.fsum(a * b)
            bound += 128 * np.abs(a).max() * np.abs(b).max()
        err = abs(float(H) + float(L) - exact) / bound
        worst = max(worst, err)
    assert worst <= 2.0 ** -38, worst
