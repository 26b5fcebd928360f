"""Matvec with A split by rows across ranks (one process per GPU).

y = A x on the compressed form (Introduction: the same operation as on the
uncompressed matrix), with A's rows split into contiguous blocks, one per
rank, and x replicated.  Every block except the last holds a multiple of 32
rows: 32 fields of b bits are b whole words (Methods, Method 1: the fields
are laid end to end), so each block of y starts on a word boundary of the
packed y at any width.  The steps, per rank:

1. y_r = A_r x, packed at its own exact width (ccm_matvec);
2. the width statistics of y_r (bit length of the OR of the folded values,
   any negative) are reduced with MAX over ranks: the width rule applied to
   the whole of y, since the bit length of an OR is the largest bit length;
3. y_r re-packed at that width into its rows of a full-size y buffer whose
   other words are zero (ccm_repack);
4. a SUM all-reduce of the word buffers (the blocks occupy disjoint words)
   leaves the packed y, header included, on every rank.

All arithmetic runs in libccm's kernels; this module only schedules the
collectives (torch.distributed: NCCL between GPUs, gloo between CPU ranks).
The backend object supplies the per-rank steps, so the same schedule runs on
the GPU library and, in tests, on any other implementation of the steps.
"""
from __future__ import annotations

import torch


def row_blocks(m: int, world: int) -> list[tuple[int, int]]:
    """Rows [r0, r1) of each rank: balanced, every block but the last a
    multiple of 32 rows (ranks past the end get empty blocks)."""
    groups = (m + 31) // 32
    per, extra = divmod(groups, world)
    out, g = [], 0
    for r in range(world):
        cnt = per + (1 if r < extra else 0)
        r0, r1 = min(m, 32 * g), min(m, 32 * (g + cnt))
        out.append((r0, r1))
        g += cnt
    return out


def width_from_stats(bitlen: int, neg: int) -> tuple[int, int]:
    """The width rule (Eq. 1, signed reading) from the bit length of the OR
    of the folded values and the any-negative flag."""
    if neg:
        return bitlen + 1, 1
    return max(1, bitlen), 0


class CcmBackend:
    """The per-rank steps on this rank's GPU through libccm."""

    def __init__(self):
        from . import ccm
        self.ccm = ccm

    def matvec(self, a, x):
        return self.ccm.matvec(a, x)

    def stats(self, y) -> tuple[int, int, int]:
        """(bit length of the OR of the folded values, any negative, status)."""
        h = y.header()
        return int(h.stat_or).bit_length(), int(h.stat_neg != 0), int(h.status)

    def repack(self, y, width: int, is_signed: int, rows: int, row_offset: int):
        out = self.ccm.PackedMatrix(rows, 1, self.ccm.words_for(rows, 1, width), y.device)
        return self.ccm.repack_into(y, width, is_signed, out, row_offset)

    def words(self, out) -> torch.Tensor:
        """The int32 word buffer (after the header) the SUM all-reduce combines."""
        return out.buf[self.ccm.HEADER_WORDS:]

    def finish(self, out):
        out._written()
        return out.check()


def sharded_matvec(a_block, x, m: int, row_offset: int, backend=None, group=None):
    """y = A x where this rank holds rows [row_offset, row_offset +
    a_block.rows) of A (m rows in all) and all of x.  Returns the packed y
    (m x 1) on every rank; a failure on any rank (an input error, int64
    overflow) raises on every rank."""
    import torch.distributed as dist
    backend = backend or CcmBackend()
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    y_r = backend.matvec(a_block, x)
    bitlen, neg, status = backend.stats(y_r)
    dev = backend.words(y_r).device
    st = torch.tensor([bitlen, neg, -status], dtype=torch.int64, device=dev)
    if world > 1:
        dist.all_reduce(st, op=dist.ReduceOp.MAX, group=group)
    if int(st[2]) != 0:
        raise RuntimeError(f"sharded matvec: a rank's block failed with status {-int(st[2])}")
    width, is_signed = width_from_stats(int(st[0]), int(st[1]))
    out = backend.repack(y_r, width, is_signed, m, row_offset)
    if world > 1:
        dist.all_reduce(backend.words(out), op=dist.ReduceOp.SUM, group=group)
    return backend.finish(out)
