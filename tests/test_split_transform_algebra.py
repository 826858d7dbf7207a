"""The factorisation behind the warp-split column stages, checked on the CPU.

The column transform of length N = 512 RB with at most 512 non-zero rows (1024 at RB = 16)
is computed as RB 512-point DFTs, one per warp: bin q = k1 + RB k2 takes the DFT k2 of
u_k1[m] = w_N^(m k1) (x[m] + w_16^(k1) x[m + 512]).  Each warp splits its DFT as 16 values
per lane (m = 32 j + l): a step-1 twiddle w_N^((32 j + 16 p) k1), a DFT16 over j, the
per-lane powers w_512^(l a), a radix-2 butterfly between lanes l and l ^ 16, the lane
constant w_32^(l' p) w_N^(l' k1), a transpose within each half-warp and a second DFT16.
This file replays exactly those steps with numpy (lanes as an array axis) and compares
them with a direct FFT, for the forward and for the conjugate-transposed adjoint chain, at
every RB the kernels are built for.  It tests the algebra the kernels implement, not the
kernels themselves (the GPU parity tests do that).
"""
import numpy as np
import pytest


def w(M, e):
    return np.exp(-2j * np.pi * np.asarray(e, dtype=np.float64) / M)


LANE = np.arange(32)
LP, P = LANE & 15, LANE >> 4


def split_forward(x, RB):
    """Bins X[q], q < 512 RB, of the zero-padded column x (len <= 512, or 1024 at RB = 16)."""
    N = 512 * RB
    xx = np.zeros(1024 if RB == 16 else 512, complex)
    xx[: len(x)] = x
    X = np.zeros(N, complex)
    j = np.arange(16)
    for k1 in range(RB):
        m = 32 * j[None, :] + LANE[:, None]                  # [lane][j]
        v = xx[m]
        if RB == 16:
            v = v + w(16, k1) * xx[m + 512]
        v = v * w(N, (32 * j[None, :] + 16 * P[:, None]) * k1)
        v = np.fft.fft(v, axis=1)                            # DFT16 over j -> a
        a = np.arange(16)
        v = v * w(512, LANE[:, None] * a[None, :])
        partner = v[LANE ^ 16]
        v = partner + np.where(P == 1, -1, 1)[:, None] * v
        v = v * w(N, LP * (k1 + 16 * RB * P))[:, None]
        # lane (l', p) writes row a + 16 p, column l'; lane L reads row L
        rows = np.zeros((32, 16), complex)
        for L in range(32):
            rows[a + 16 * P[L], LP[L]] = v[L]
        v = np.fft.fft(rows, axis=1)                         # DFT16 over l' -> b
        b = np.arange(16)
        for L in range(32):
            X[k1 + RB * (L + 32 * b)] = v[L]
    return X


def split_adjoint(Z, RB, n_out):
    """z[m] = sum_q Z[q] w_N^(-m q), m < n_out, by the conjugate-transposed chain per warp and the
    sum of the RB partial rows in the order k1 = 0, 1, ..."""
    N = 512 * RB
    z = np.zeros(1024 if RB == 16 else 512, complex)
    b = np.arange(16)
    a = np.arange(16)
    j = np.arange(16)
    for k1 in range(RB):
        v = np.stack([Z[k1 + RB * (L + 32 * b)] for L in range(32)])          # [L][b]
        rows = np.fft.ifft(v, axis=1) * 16                                      # -> l'
        v = np.stack([rows[a + 16 * P[L], LP[L]] for L in range(32)])          # lane (l', p) [a]
        v = v * np.conj(w(N, LP * (k1 + 16 * RB * P)))[:, None]
        partner = v[LANE ^ 16]
        v = partner + np.where(P == 1, -1, 1)[:, None] * v
        v = v * np.conj(w(512, LANE[:, None] * a[None, :]))
        v = np.fft.ifft(v, axis=1) * 16                                         # -> j
        v = v * np.conj(w(N, (32 * j[None, :] + 16 * P[:, None]) * k1))
        s = np.zeros(512, complex)
        for L in range(32):
            s[32 * j + L] = v[L]
        z[:512] += s
        if RB == 16:
            z[512:] += np.conj(w(16, k1)) * s
    return z[:n_out]


@pytest.mark.parametrize("RB,rows", [(1, 64), (2, 128), (4, 255), (8, 512), (8, 220), (16, 553), (16, 1024)])
def test_split_forward_equals_fft(RB, rows):
    rng = np.random.default_rng(RB * 1000 + rows)
    x = rng.standard_normal(rows) + 1j * rng.standard_normal(rows)
    X = split_forward(x, RB)
    xp = np.zeros(512 * RB, complex)
    xp[:rows] = x
    ref = np.fft.fft(xp)
    assert np.max(np.abs(X - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("RB,rows", [(1, 64), (2, 128), (4, 255), (8, 512), (16, 553), (16, 1024)])
def test_split_adjoint_is_the_transposed_transform(RB, rows):
    N = 512 * RB
    rng = np.random.default_rng(7 + RB)
    Z = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    z = split_adjoint(Z, RB, rows)
    ref = (np.fft.ifft(Z) * N)[:rows]
    assert np.max(np.abs(z - ref)) <= 1e-12 * np.max(np.abs(ref))
    # <F x, Z> = <x, F^H Z> for the zero-padded forward restricted to `rows` inputs
    x = rng.standard_normal(rows) + 1j * rng.standard_normal(rows)
    lhs = np.vdot(split_forward(x, RB), Z)
    rhs = np.vdot(x, z)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_half_warp_transpose_is_conflict_free():
    """The transpose's slots (rows of 17): the 16 lanes of a half-warp hit 16 distinct 8-byte
    banks on the write (lanes l', fixed a) and on the read (lanes L, fixed l'), and every slot
    stays inside the warp's 544-slot region."""
    slots_written = set()
    for a in range(16):
        for p in range(2):
            s = [17 * (a + 16 * p) + lp for lp in range(16)]
            assert len({x % 16 for x in s}) == 16
            slots_written.update(s)
    for lp in range(16):
        for half in range(2):
            s = [17 * L + lp for L in range(16 * half, 16 * half + 16)]
            assert len({x % 16 for x in s}) == 16
    assert max(slots_written) < 544 and len(slots_written) == 512
