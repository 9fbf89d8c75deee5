"""The digit slicing behind the tensor-core products, emulated in IEEE binary32
with numpy (no GPU): the invariants the exactness argument rests on.

A double-float value (h, l) of a row whose entries lie below 2^e is written as
seven signed base-256 digits of (h + l) 2^(7-e): each step takes the nearest
integer of the remainder's high part, subtracts it exactly, renormalises the
remainder with an error-free sum and scales it by 256.  Checked here:
  * every digit is an integer with |d| <= 128 (so d 2^(-8i) is exact in bf16),
  * the digits reconstruct h + l to within 2^(e-56) (the dropped remainder),
  * the per-level sums of the five exact levels stay below 2^24 for the worst
    digits and the deepest group (96 complex = 192 real inner entries)."""
import numpy as np

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def digits(h, l, e, S=7):
    sc = f32(2.0 ** (7 - e))
    x, y = f32(h * sc), f32(l * sc)
    out = []
    for _ in range(S):
        d = f32(np.rint(f32(x + y)))
        out.append(d)
        s2, e2 = two_sum(f32(x - d), y)
        x, y = f32(s2 * f32(256.0)), f32(e2 * f32(256.0))
    return out


def to_df(v):
    h = f32(v)
    return h, f32(v - float(h))


def bf16_exact(v):
    b = np.array([v], dtype=np.float32).view(np.uint32)[0]
    return (b & 0xFFFF) == 0


def test_digits_are_bounded_exact_and_reconstruct():
    rng = np.random.default_rng(0)
    for trial in range(3000):
        e = int(rng.integers(-20, 20))
        mag = 2.0 ** e * (1 - 2.0 ** -30) * rng.random() ** rng.integers(1, 6)
        v = mag * rng.choice([-1.0, 1.0])
        h, l = to_df(v)
        if abs(float(h)) >= 2.0 ** e:            # the row scale bounds the high parts
            continue
        ds = digits(h, l, e)
        acc = 0.0
        for i, d in enumerate(ds):
            assert float(d) == int(d) and abs(int(d)) <= 128, (v, e, ds)
            w = f32(2.0 ** (-8 * i))
            assert bf16_exact(f32(d * w))       # the tile value d 2^(-8i) is a bf16
            acc += float(d) * 2.0 ** (e - 7 - 8 * i)
        assert abs(acc - (float(h) + float(l))) <= 2.0 ** (e - 56), (v, e, acc)


def test_row_maximum_itself_and_ties():
    # entries at the top of the range and exactly on half-integers of a digit
    for e in (0, 3, -7):
        for v in (2.0 ** e * (1 - 2.0 ** -24), -(2.0 ** e) * (1 - 2.0 ** -24), 2.0 ** (e - 8) * 0.5,
                  2.0 ** (e - 7) * 127.5, -(2.0 ** (e - 7)) * 128.5 / 2):
            h, l = to_df(v)
            ds = digits(h, l, e)
            assert all(abs(int(d)) <= 128 for d in ds)
            rec = sum(float(d) * 2.0 ** (e - 7 - 8 * i) for i, d in enumerate(ds))
            assert abs(rec - (float(h) + float(l))) <= 2.0 ** (e - 56)


def test_exact_levels_fit_binary32():
    # level l (< 5) holds (l + 1) digit pairs per real inner entry, each product
    # an integer multiple of 2^(-8 l) of magnitude <= 128^2; a group has at most
    # 192 real inner entries (96 complex in the 2 x 2 block form)
    for lev in range(5):
        worst = (lev + 1) * 192 * 128 * 128
        assert worst < 2 ** 24, (lev, worst)
    # the merged accumulator starts at level 5: below 2^-40 of the level-0 scale
    assert 2.0 ** (-8 * 5) <= 2.0 ** -40
