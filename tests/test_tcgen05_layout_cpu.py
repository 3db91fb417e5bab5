"""The tcgen05 sweep's data flow for one block, replayed on the CPU: digit
planes, Toeplitz and Hankel digit matrices and sheared planes written at the
byte offsets of the library's tiled layout (w2_debug_umma_tile_off), every MMA
operand read back through the no-swizzle canonical layout with the strides
the sweep passes to its descriptors (the convention the GPU self-test
confirmed: leading offset = K-direction core-matrix stride, stride offset =
M/N-direction), the digit-stacked one-body chains and the two-body chains
accumulated as the tensor core would (exact integers), and the epilogue's
int64 recombination.  The result must equal Theta written from its
definition (the three Toeplitz sums of Eq. Hartree_FSM / two_body_FSM) to
FP64 rounding, and every operand read must stay inside its region.  No
device is used."""
import struct

import numpy as np
import pytest

from paper_2511_11354_gb300 import build as w2build
from paper_2511_11354_gb300 import w2

NK = 64
MAT, HMAT, GMAT = NK * NK * 2, 15 * 128, 2 * NK * NK * 2
OFF_F = 0
OFF_T1 = OFF_F + 7 * MAT
OFF_B2 = OFF_T1 + 7 * MAT
OFF_H = OFF_B2 + 6 * MAT
OFF_G = OFF_H + 12 * HMAT
OFF_MISC = OFF_G + 2 * GMAT


@pytest.fixture(scope="module")
def toff():
    w2build.build()
    t64 = np.array([[w2.umma_tile_off(r, c, 64) for c in range(64)] for r in range(64)], dtype=np.int64)
    t128 = np.array([[w2.umma_tile_off(r, c, 128) for c in range(128)] for r in range(64)], dtype=np.int64)
    return t64, t128


def digits6(v, emax):
    """Six balanced base-256 digits of |v| 2^(48 - E), 2^E = 2^(emax - 1022), with v's sign."""
    b = struct.unpack("<Q", struct.pack("<d", float(v)))[0]
    e = (b >> 52) & 0x7FF
    m = (b & 0xFFFFFFFFFFFFF) | ((1 << 52) if e else 0)
    sh = emax - (e if e else 1) + 5
    n = (m + (1 << (sh - 1))) >> sh if sh < 64 else 0
    d = [0] * 6
    for s in range(5, 0, -1):
        lo = n & 255
        d[s] = lo - ((lo & 128) << 1)
        n = (n - d[s]) >> 8
    d[0] = n
    return [-x for x in d] if b >> 63 else d


def expo(v):
    return (struct.unpack("<Q", struct.pack("<d", float(v)))[0] >> 52) & 0x7FF


def operand(sm, start, lbo, sbo, mn, rows):
    """rows x 16 values of an MMA operand (16-bit integers) read from the canonical layout."""
    i = np.arange(rows)[:, None]
    k = np.arange(16)[None, :]
    if mn:
        off = start + (i // 8) * sbo + (k // 8) * lbo + (k % 8) * 16 + (i % 8) * 2
    else:
        off = start + (i // 8) * sbo + (k // 8) * lbo + (i % 8) * 16 + (k % 8) * 2
    assert off.min() >= 0 and off.max() + 2 <= OFF_MISC
    return sm[off // 2].astype(np.float64)


def theta_by_the_sweep(F, K1, K2, K12, toff):
    t64, t128 = toff
    ef = max(expo(x) for x in F.ravel())
    ek = max(expo(x) for x in np.concatenate([K1, K2, K12]))
    emax, kmax = max(ef, 1), max(ek, 1)
    sm = np.zeros(OFF_MISC // 2, dtype=np.int64)  # 16-bit words, holding the digits as integers
    dF = np.array([[digits6(F[r, c], emax) for c in range(NK)] for r in range(NK)])  # [r][c][s]
    for s in range(6):
        sm[(OFF_F + (s + 1) * MAT + t64) // 2] = dF[:, :, s]
    dK = [np.array([digits6(x, kmax) for x in row]) for row in (K1, K2, K12)]  # [j][t]
    r = np.arange(NK)[:, None]
    k = np.arange(NK)[None, :]
    for t in range(6):  # Toeplitz M[r][k] = K(k - r): A1 after the zero matrix, B2
        sm[(OFF_T1 + (t + 1) * MAT + t64) // 2] = dK[0][k - r + 63, t]
        sm[(OFF_B2 + t * MAT + t64) // 2] = dK[1][k - r + 63, t]
    core = np.arange(15)[:, None, None]
    bb = np.arange(8)[None, :, None]
    aa = np.arange(8)[None, None, :]
    hoff = core * 128 + bb * 16 + aa * 2
    for t in range(6):  # Hankel: core q, row b, entry a = K12(63 - 8q - a - b); H' carries 2^-8
        vals = dK[2][126 - 8 * core - aa - bb, t]
        sm[(OFF_H + t * HMAT + hoff) // 2] = vals
        sm[(OFF_H + (6 + t) * HMAT + hoff) // 2] = vals  # scaled copy: the 2^-8 is applied below
    acc = np.zeros((128, 512))

    def mma(col, a, b, accumulate, scale=1.0):
        d = (a @ b.T) * scale
        if accumulate:
            acc[:, col:col + 64] += d
        else:
            acc[:, col:col + 64] = d

    for s in range(6):  # T1 dominoes
        ts = -1 if s & 1 else 0
        while s + ts <= 4:
            for kc in range(4):
                a = operand(sm, OFF_T1 + (ts + 1) * MAT + 256 * kc, 128, 1024, False, 128)
                b = operand(sm, OFF_F + (s + 1) * MAT + 2048 * kc, 1024, 128, True, 64)
                mma(32 * (s + ts), a, b, not (s == 0 and kc == 0))
            ts += 2
    for t in range(6):  # T2 dominoes
        ss = -1 if t & 1 else 0
        while ss + t <= 4:
            for kc in range(4):
                a = operand(sm, OFF_F + (ss + 1) * MAT + 256 * kc, 128, 1024, False, 128)
                b = operand(sm, OFF_B2 + t * MAT + 256 * kc, 128, 1024, False, 64)
                mma(32 * (ss + t), a, b, True)
            ss += 2
    kp = np.arange(64)[:, None]
    c = np.arange(128)[None, :]
    for s in range(6):  # sheared plane G_s[c][k'] = F_s[63 - k'][c - 63 + k'], then the two-body chains
        m = c - 63 + kp
        vals = np.where((m >= 0) & (m < NK), dF[63 - kp, np.clip(m, 0, NK - 1), s], 0)
        sm[(OFF_G + (s & 1) * GMAT + t128) // 2] = vals
        for t in range(6 - s):
            d = s + t
            h = OFF_H + ((6 + t) if d == 5 else t) * HMAT
            for kc in range(4):
                a = operand(sm, OFF_G + (s & 1) * GMAT + 4096 * kc, 2048, 128, True, 128)
                b = operand(sm, h + 256 * kc, 128, 128, False, 64)
                mma(192 + 64 * min(d, 4), a, b, not (s == 0 and t <= 4 and kc == 0), 2.0 ** -8 if d == 5 else 1.0)
    # epilogue: units of 2^4 diagonal-5 units
    I = [[0] * NK for _ in range(NK)]
    for L in range(128):
        top, n1 = L < 64, L & 63
        for n2 in range(NK):
            v = 0
            for e in range(3):
                q = int(round(acc[L, 64 * e + n2]))
                v += q << (8 * (4 - 2 * e) + 4) if top else (q << (8 * (3 - 2 * e) + 4) if e < 2 else (q + 8) >> 4)
            I[n1][n2] += v
    for cc in range(128):
        for n1 in range(NK):
            v = sum(int(round(acc[cc, 192 + 64 * d + n1])) << (8 * (4 - d) + 4) for d in range(4))
            v += int(np.rint(np.float32(acc[cc, 448 + n1]) * 16))
            n2 = cc - n1
            if 0 <= n2 < NK:
                I[n1][n2] += v
    xs = emax + kmax - 2096
    return np.array([[float(I[a][b]) * 2.0 ** xs for b in range(NK)] for a in range(NK)])


def theta_by_definition(F, K1, K2, K12):
    n = np.arange(NK)
    T1 = np.array([[K1[n - a + 63] @ F[:, b] for b in range(NK)] for a in range(NK)])
    T2 = np.array([[F[a, :] @ K2[n - b + 63] for b in range(NK)] for a in range(NK)])
    T12 = np.zeros((NK, NK))
    for a in range(NK):
        for b in range(NK):
            kk = n[(a + b - n >= 0) & (a + b - n < NK)]
            T12[a, b] = K12[kk - a + 63] @ F[kk, a + b - kk]
    return T1 + T2 + T12


@pytest.mark.parametrize("seed", [0, 1])
def test_sweep_layout_reproduces_theta(toff, seed):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((NK, NK)) * np.exp(rng.uniform(-4, 4, (NK, NK)))
    K1, K2 = rng.standard_normal(127), rng.standard_normal(127)
    K12 = 3.0 * rng.standard_normal(127)
    got = theta_by_the_sweep(F, K1, K2, K12, toff)
    ref = theta_by_definition(F, K1, K2, K12)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_a_transposed_operand_fails(toff):
    """A planted mistake (the T1 Toeplitz digits written transposed, K(r - k))
    must be caught."""
    rng = np.random.default_rng(3)
    F = rng.standard_normal((NK, NK))
    K1, K2, K12 = (rng.standard_normal(127) for _ in range(3))
    ref = theta_by_definition(F, K1, K2, K12)
    bad = theta_by_the_sweep(F, K1[::-1].copy(), K2, K12, toff)  # K1(j) -> K1(-j): the transposed Toeplitz
    assert np.linalg.norm(bad - ref) / np.linalg.norm(ref) > 1e-3
