"""Element-wise comparison of GPU gradients with the oracle's BF16-storage-emulated backward.

Each gradient entry is a sum over the batch, dW_l[i, j] = sum_b delta_l[b, i] A_l[b, j] (and
db_l[i] = sum_b delta_l[b, i]).  The GPU and the emulated oracle store the same values in BF16;
they differ only by FP32-vs-FP64 accumulation (relative ~1e-6 of the term magnitudes) and by
values that sit on a BF16 rounding boundary and round the other way (one BF16 unit, at most
2^-7 of the value).  So every entry must lie within 2^-7 of the sum of its terms' magnitudes,
|g - g_o| <= 2^-7 (|delta|^T |A|).  The bound is informative: for most entries the oracle's
gradient itself is larger than the bound, so a zeroed, swapped or transposed block fails.
"""
import numpy as np

C = 2.0 ** -7


def check_layer(gw, gb, ow, ob, delta, act, what=""):
    bound_w = C * (np.abs(delta).T @ np.abs(act)) + 1e-30
    bound_b = C * np.abs(delta).sum(axis=0) + 1e-30
    bad = np.abs(gw - ow) > bound_w
    assert not bad.any(), (what, int(bad.sum()), np.argwhere(bad)[:5])
    assert (np.abs(gb - ob) <= bound_b).all(), what
    live = bound_w > 1e-29
    assert (np.abs(ow)[live] > bound_w[live]).mean() > 0.5, what
