"""Which cells of a span segmentation (Sec. II-C) a bounded error of the span spectra cannot
change: test infrastructure shared by the GPU decomposition tests and their CPU check."""
import numpy as np


def decisive_cells(refs, threshold, err):
    """Cells whose segmentation (the threshold test of every span and the choice among the
    passing spans) cannot change when each span's spectrum moves by at most err[h] in absolute
    value.  A power p = |X|^2 then moves by at most 2|X| e + e^2, and the threshold
    thr^2 max p by thr^2 times that bound at the maximum.  A cell is decisive when every span
    is clear of the threshold by more than both bands, and, among the spans above it, the
    largest power is clear of the runner-up by more than their two bands."""
    p = np.abs(refs) ** 2
    band = 2.0 * np.abs(refs) * err[:, None, None, None] + (err ** 2)[:, None, None, None]
    hmax = int(np.argmax(p.reshape(len(refs), -1).max(axis=1)))
    pmax = p[hmax].max()
    floor = threshold * threshold * pmax
    band_floor = threshold * threshold * (2.0 * np.sqrt(pmax) * err[hmax] + err[hmax] ** 2)
    above = p - band > floor + band_floor
    below = p + band < floor - band_floor
    near_floor = ~(above | below).all(axis=0)
    pc = np.where(above, p, -np.inf)
    order = np.argsort(-pc, axis=0)
    p1 = np.take_along_axis(pc, order[:1], 0)[0]
    b1 = np.take_along_axis(band, order[:1], 0)[0]
    if len(refs) > 1:
        p2 = np.take_along_axis(pc, order[1:2], 0)[0]
        b2 = np.take_along_axis(band, order[1:2], 0)[0]
        with np.errstate(invalid="ignore"):  # cells with no span above the threshold: -inf - -inf
            near_tie = np.isfinite(p2) & ((p1 - p2) <= b1 + b2)
    else:
        near_tie = np.zeros(p1.shape, bool)
    return ~(near_floor | near_tie)
