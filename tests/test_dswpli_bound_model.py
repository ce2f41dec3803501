"""The error bound behind the mixed full window's DSWPLI tolerance (CPU, no GPU).

The mixed-precision full window sums Im, |Im| and Im^2 of a pair-bin in FP32 over chunks of
at most 36 trials (Im^2 by fused multiply-add) and adds each chunk's partial sums into
FP64-class window sums; DSWPLI = ((sum Im)^2 - sum Im^2) / ((sum |Im|)^2 - sum Im^2) is then
formed from those. The bound the GPU tests use per bin is
6 m u (sum |Im|)^2 / ((sum |Im|)^2 - sum Im^2), m = min(K, 36), u = 2^-24. Here that
arithmetic is emulated exactly (FP32 roundings via numpy float32, the fused square as an
exact FP64 product rounded once) and compared with FP64 on windows of 2 to 100 trials,
including two-trial windows where one term dominates, where the bound is largest.
"""

import numpy as np

U = 2.0 ** -24
NK = 36


def emulated_dswpli(im):
    """DSWPLI of one pair-bin from FP32 chunk sums promoted to FP64 window sums."""
    im = np.asarray(im, np.float32)
    K = im.shape[0]
    nchunk = -(-K // NK)
    csize = -(-K // nchunk)
    s = a = q = 0.0  # window sums (FP64 stands in for the double words)
    for c0 in range(0, K, csize):
        pim = pab = psq = np.float32(0.0)
        for t in im[c0:c0 + csize]:
            pim = np.float32(pim + t)
            pab = np.float32(pab + abs(t))
            psq = np.float32(np.float64(t) * np.float64(t) + np.float64(psq))  # fused: one rounding
        s += float(pim)
        a += float(pab)
        q += float(psq)
    nz = int(np.count_nonzero(im))
    if nz <= 1:
        return 0.0
    num, den = s * s - q, a * a - q
    return num / den if den != 0 else 0.0


def exact_dswpli(im):
    im = np.asarray(im, np.float64)
    s, a, q = im.sum(), np.abs(im).sum(), (im * im).sum()
    den = a * a - q
    return ((s * s - q) / den if den != 0 else 0.0), a, den


def test_dswpli_error_within_the_derived_bound():
    rng = np.random.default_rng(7)
    worst = 0.0
    for K in (2, 2, 2, 3, 5, 36, 37, 100):
        for _ in range(400):
            im = rng.standard_normal(K) * np.exp2(rng.uniform(-12, 0, K) * (K <= 3))  # spread for tiny K
            im = im.astype(np.float32)
            ref, a, den = exact_dswpli(im)
            if den <= 0:
                continue
            got = emulated_dswpli(im)
            bound = 6 * min(K, NK) * U * a * a / den
            assert abs(got - ref) <= bound + 1e-12, (K, got, ref, bound)
            worst = max(worst, abs(got - ref) / bound)
    assert worst > 1e-3  # the bound is not vacuous: errors reach a visible fraction of it


def test_two_trials_one_dominant_term_is_ill_conditioned():
    # K = 2, opposite signs, |Im_1 / Im_2| = 2^15: DSWPLI is exactly -1; sum Im and sum |Im|
    # round differently in FP32, and the debiased differences (2 Im_1 Im_2 each) are tiny
    # beside the squares they come from (with equal signs both sums round alike and the
    # ratio stays exactly 1)
    im = np.array([1.0, -(2.0 ** -15) * 1.37], np.float32)
    ref, a, den = exact_dswpli(im)
    assert abs(ref + 1.0) < 1e-12
    got = emulated_dswpli(im)
    bound = 6 * 2 * U * a * a / den
    assert 1e-3 < abs(got - ref) <= bound  # 1.5e-3 against a bound of 8.6e-3
