"""The split FP16 representation of the tensor-core operands (CPU, numpy's IEEE binary16 as the
emulation): a deviation v (nm) is scaled by 2^8 and split v' = h + l, h = fp16(v'),
l = fp16(v' - h); a product is formed as h h' + h l' + l h', with l l' dropped.

Checked here, from the IEEE formats alone:
  * h + l is within 2^-22 of v' for |v| >= 5e-4 nm, although l is then mostly subnormal
    (the absolute spacing 2^-24 of FP16 subnormals bounds the error of l);
  * below that the bound fails (the scale was chosen for deviations of at least ~5e-4 nm);
  * the three-product form is within 3 * 2^-22 of v' w' (representation errors of both
    operands and the dropped l l', each at most 2^-22 relative);
  * deviations below 255.9 nm stay finite (2^8 * 255.9 < 65504, the largest FP16), 256 nm does not.
"""
import numpy as np


def _split(v):
    vs = (np.asarray(v, dtype=np.float64) * 256.0).astype(np.float32)
    h = vs.astype(np.float16)
    l = (vs - h.astype(np.float32)).astype(np.float16)
    return vs.astype(np.float64), h.astype(np.float64), l.astype(np.float64)


def _deviations(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n)) * rng.choice([-1.0, 1.0], n)


def test_split_carries_22_bits_above_5e4_nm():
    rng = np.random.default_rng(11)
    for lo, hi in [(5e-4, 1e-3), (1e-3, 1.0), (1.0, 255.0)]:
        vs, h, l = _split(_deviations(rng, lo, hi, 400_000))
        rel = np.abs(h + l - vs) / np.abs(vs)
        assert rel.max() <= 2.0**-22, (lo, hi, rel.max())
    # just above the threshold l is subnormal almost always: the bound does not need it normal
    vs, h, l = _split(_deviations(rng, 5e-4, 1e-3, 100_000))
    assert np.mean(np.abs(l) < 2.0**-14) > 0.9


def test_split_loses_bits_below_the_threshold():
    rng = np.random.default_rng(12)
    vs, h, l = _split(_deviations(rng, 1e-5, 1e-4, 100_000))
    assert (np.abs(h + l - vs) / np.abs(vs)).max() > 2.0**-22


def test_three_products_within_three_units_of_2_22():
    rng = np.random.default_rng(13)
    a = _deviations(rng, 5e-4, 50.0, 400_000)
    b = _deviations(rng, 5e-4, 50.0, 400_000)
    va, ha, la = _split(a)
    vb, hb, lb = _split(b)
    three = ha * hb + ha * lb + la * hb  # exact in float64: FP16 products carry 22 bits
    rel = np.abs(three - va * vb) / np.abs(va * vb)
    assert rel.max() <= 3 * 2.0**-22, rel.max()
    # the dropped product is the largest single term of the error budget's size
    assert (np.abs(la * lb) / np.abs(va * vb)).max() <= 2.0**-22


def test_largest_finite_deviation():
    _, h, _ = _split([255.9, -255.9])
    assert np.all(np.isfinite(h))
    with np.errstate(over="ignore"):
        _, h, _ = _split([256.0])
    assert not np.isfinite(h[0])
