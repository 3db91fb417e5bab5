"""The tcgen05 encoders of the library, bit by bit, on the CPU (no device use):
the shared-memory matrix descriptor and the kind::f16 instruction descriptor
against the field tables of the PTX ISA (tcgen05 "matrix descriptor" and
"instruction descriptor" sections), and the tiled operand layout against the
no-swizzle canonical layout (8 x 8 core matrices of 128 contiguous bytes)."""
import numpy as np
import pytest

from paper_2511_11354_gb300 import build as w2build
from paper_2511_11354_gb300 import w2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    w2build.build()


def field(v, lo, width):
    return (v >> lo) & ((1 << width) - 1)


@pytest.mark.parametrize("saddr,lbo,sbo", [(0, 128, 1024), (1024, 1024, 128), (16, 16, 16),
                                           (227 * 1024 - 16, 2048, 256), (0x3fff0, 0x3fff0, 0x3fff0),
                                           (49152 + 256, 128, 8192)])
def test_smem_descriptor_fields(saddr, lbo, sbo):
    d = w2.umma_smem_desc(saddr, lbo, sbo)
    assert field(d, 0, 14) == saddr >> 4          # start address, 16-byte units
    assert field(d, 14, 2) == 0
    assert field(d, 16, 14) == lbo >> 4           # leading-dimension byte offset
    assert field(d, 30, 2) == 0
    assert field(d, 32, 14) == sbo >> 4           # stride-dimension byte offset
    assert field(d, 46, 3) == 0b001               # fixed constant
    assert field(d, 49, 3) == 0                   # matrix base offset
    assert field(d, 52, 1) == 0                   # leading-dimension mode: byte offset
    assert field(d, 53, 8) == 0
    assert field(d, 61, 3) == 0                   # no swizzle


def test_smem_descriptor_fields_random():
    rng = np.random.default_rng(5)
    for _ in range(200):
        s, l, t = (int(x) * 16 for x in rng.integers(0, 1 << 14, 3))
        d = w2.umma_smem_desc(s, l, t)
        want = (s >> 4) | ((l >> 4) << 16) | ((t >> 4) << 32) | (1 << 46)
        assert d == want


@pytest.mark.parametrize("M", [64, 128])
@pytest.mark.parametrize("a_mn,b_mn", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_instruction_descriptor_fields(M, a_mn, b_mn):
    for N in range(16, 257, 16):
        i = w2.umma_idesc(M, N, a_mn, b_mn)
        assert field(i, 0, 2) == 0                # sparsity selector
        assert field(i, 2, 1) == 0                # dense
        assert field(i, 3, 1) == 0                # no saturation
        assert field(i, 4, 2) == 1                # D: F32
        assert field(i, 6, 1) == 0
        assert field(i, 7, 3) == 1                # A: BF16
        assert field(i, 10, 3) == 1               # B: BF16
        assert field(i, 13, 1) == 0 and field(i, 14, 1) == 0   # no negation
        assert field(i, 15, 1) == a_mn            # A major-ness
        assert field(i, 16, 1) == b_mn            # B major-ness
        assert field(i, 17, 6) == N >> 3
        assert field(i, 23, 1) == 0
        assert field(i, 24, 5) == M >> 4
        assert field(i, 29, 3) == 0               # reserved, maximum shift 0


@pytest.mark.parametrize("rows,cols", [(64, 64), (128, 64), (64, 16), (16, 128)])
def test_tiled_layout_is_the_canonical_core_matrix_layout(rows, cols):
    off = np.array([[w2.umma_tile_off(r, c, cols) for c in range(cols)] for r in range(rows)])
    # a bijection onto the 2 rows cols bytes, 2-byte aligned
    assert sorted(off.ravel().tolist()) == list(range(0, 2 * rows * cols, 2))
    for r0 in range(0, rows, 8):
        for c0 in range(0, cols, 8):
            core = off[r0:r0 + 8, c0:c0 + 8]
            base = core[0, 0]
            assert base % 128 == 0                                   # 128 contiguous bytes
            assert np.array_equal(core - base, np.arange(64).reshape(8, 8) * 2)  # row r at byte 16 r
            assert base == ((r0 // 8) * (cols // 8) + c0 // 8) * 128  # tiles row-major
