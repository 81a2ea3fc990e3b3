"""Host checks of constant tables that the CUDA kernels embed (no GPU).

The block-per-warp GMM backward at D = 128 deals the 120 off-diagonal 8x8
blocks of the lower triangle to 15 warps of eight (table kOffBlocks16). Every
block must appear exactly once (otherwise a part of S_k would be missing or
counted twice), and within a warp the distinct row chunks, and the distinct
column chunks, must differ mod 8 so that the warp's 16-byte shared loads fall
in different bank groups."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2104_05372_b300", "csrc", "gmm_kernels.cuh")


def _table():
    src = open(SRC).read()
    m = re.search(r"kOffBlocks16\[120\]\s*=\s*\{([^}]*)\}", src)
    assert m, "kOffBlocks16 not found"
    return [int(v, 16) for v in re.findall(r"0x[0-9a-fA-F]+", m.group(1))]


def test_off_diagonal_table_covers_every_block_once():
    blocks = [(v >> 4, v & 15) for v in _table()]
    assert len(blocks) == 120
    assert sorted(blocks) == sorted((a, b) for a in range(16) for b in range(a))


def test_off_diagonal_table_warps_are_bank_conflict_free():
    blocks = [(v >> 4, v & 15) for v in _table()]
    for w in range(15):
        group = blocks[8 * w:8 * w + 8]
        for side in (0, 1):
            chunks = {blk[side] for blk in group}
            assert len({c % 8 for c in chunks}) == len(chunks), (w, group)
