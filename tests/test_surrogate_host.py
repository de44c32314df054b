"""CPU: the host-side logic of the surrogate -- the output layout built from a
march's norms and snapshots, the carrier taken out of the amplitude, feature
normalisation and the seeded draws (no GPU work)."""
import numpy as np

import workloads as W
from paper_1707_05943_gb300 import surrogate as S


def test_targets_layout_and_carrier():
    w = W.surrogate_draw(5, 1)[0][0]
    nt, nx = w.nt, w.nx
    norms = np.arange(nt, dtype=np.float64) * 1e-3
    # snapshots of a pure carrier psi = A exp(i k ((x + a) - 2 t)) (rows 0, 16, 32, ...)
    rows = np.arange(nt // 16)
    xa = (np.arange(nx) + 1) * w.delta
    t = 16 * rows * w.delta
    amp = 0.3 - 0.1j
    snaps = (amp * np.exp(1j * w.k * (xa[None, :] - 2 * t[:, None]))).astype(np.complex64)
    y = S.targets_from_march(norms, snaps, w)
    assert y.shape == (S.N_OUT,)
    assert np.array_equal(y[:S.N_TIMES], norms[0:2 * S.N_TIMES:2])
    z = y[S.N_TIMES:].reshape(S.AMP_ROWS, S.AMP_COLS, 2)
    # the carrier is divided out: a constant remains (to complex64 rounding of the phase)
    assert np.allclose(z[..., 0], amp.real, atol=2e-4) and np.allclose(z[..., 1], amp.imag, atol=2e-4)


def test_targets_pick_the_documented_columns():
    w = W.surrogate_draw(6, 1)[0][0]
    snaps = np.zeros((w.nt // 16, w.nx), np.complex64)
    snaps[3, 16 * 5 + 15] = 1.0  # row 48, column of x + a = 96 delta
    y = S.targets_from_march(np.zeros(w.nt), snaps, w)
    z = y[S.N_TIMES:].reshape(S.AMP_ROWS, S.AMP_COLS, 2)
    mag = np.hypot(z[..., 0], z[..., 1])
    assert np.argwhere(mag > 0.5).tolist() == [[3, 5]]
    assert abs(mag[3, 5] - 1.0) < 1e-6


def test_normalise_maps_ranges_to_unit_box():
    lo = [r[0] for r in W.SURR_RANGES]
    hi = [r[1] for r in W.SURR_RANGES]
    x = S.normalise([lo, hi], W.SURR_RANGES)
    assert np.allclose(x, [[-1] * 4, [1] * 4])


def test_draws_are_seeded_and_in_range():
    a, fa = W.surrogate_draw(17071, 64)
    b, fb = W.surrogate_draw(17071, 64)
    assert fa == fb and [w.name for w in a] == [w.name for w in b]
    f = np.array(fa)
    for i, (lo, hi) in enumerate(W.SURR_RANGES):
        slack = W.SURR_DELTA if i == 0 else 0.0  # Gamma a is rounded to a whole D
        assert np.all(f[:, i] >= lo - slack) and np.all(f[:, i] <= hi + slack)
    for w, (ga, k0a, sig, s) in zip(a, fa):
        assert w.D % 2 == 0 and abs(w.a - ga) < 1e-12
        assert abs(w.center - (-w.a - 6 * sig - s)) < 1e-9
        assert w.nx == W.SURR_NX and w.nt == W.SURR_NT
