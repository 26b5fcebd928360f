"""Row-sharded matvec (paper_1303_0270_gb300.shard) on two CPU ranks over
gloo: the schedule (block split, MAX of the width statistics, re-pack at the
agreed width into disjoint words, SUM of the word buffers) with the per-rank
steps done by the oracle, checked word for word against the oracle's matvec
of the whole matrix (integer work: tolerance 0)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleBackend:
    """The per-rank steps on the CPU: the oracle's matvec and pack."""

    def matvec(self, a, x):
        return oracle.matvec(a, x)

    def stats(self, y):
        v = oracle.unpack(y).ravel()
        orv = 0
        for e in v.tolist():
            orv |= e if e >= 0 else ~e
        return orv.bit_length(), int((v < 0).any()), 0

    def repack(self, y, width, is_signed, rows, row_offset):
        v = oracle.unpack(y).ravel()
        blk = oracle.pack_at(v, v.size, 1, width, is_signed).words
        full = np.zeros(oracle.words_for(rows, width), dtype=np.uint32)
        w0 = row_offset * width // 32
        nb = (v.size * width + 31) // 32
        full[w0:w0 + nb] = blk[:nb]
        return {"words": torch.from_numpy(full.view(np.int32).copy()), "width": width,
                "signed": is_signed, "rows": rows}

    def words(self, out):
        return out["words"] if isinstance(out, dict) else torch.zeros(1, dtype=torch.int32)

    def finish(self, out):
        return out


def _case(seed, m, n, b):
    a = synth.uniform_signed(seed, synth.STREAM_A, m * n, b).reshape(m, n)
    x = synth.uniform_int(seed, synth.STREAM_X, n, -128, 127).reshape(n, 1)
    return a, x


def _worker(rank, world, port, cases, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1303_0270_gb300 import shard
    res = []
    for seed, m, n, b in cases:
        a, x = _case(seed, m, n, b)
        r0, r1 = shard.row_blocks(m, world)[rank]
        out = shard.sharded_matvec(oracle.pack(a[r0:r1]), oracle.pack(x), m, r0,
                                   backend=OracleBackend())
        res.append((out["width"], out["signed"], out["words"].numpy().view(np.uint32).copy()))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, res))


# ragged last blocks, a block of one row, widths 1..20, y signed and unsigned
CASES = [(11, 100, 37, 5), (12, 64, 200, 12), (13, 33, 9, 1), (14, 257, 64, 20)]


def test_sharded_matvec_two_ranks_matches_oracle():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, CASES, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for i, (seed, m, n, b) in enumerate(CASES):
        a, x = _case(seed, m, n, b)
        expect = oracle.matvec(oracle.pack(a), oracle.pack(x))
        for r in (0, 1):
            width, signed, words = res[r][i]
            assert (width, signed) == (expect.width, expect.is_signed), (seed, r)
            assert np.array_equal(words, expect.words), (seed, r)


def test_row_blocks():
    from paper_1303_0270_gb300 import shard
    assert shard.row_blocks(100, 2) == [(0, 64), (64, 100)]
    assert shard.row_blocks(33, 2) == [(0, 32), (32, 33)]
    assert shard.row_blocks(10, 4) == [(0, 10), (10, 10), (10, 10), (10, 10)]
    for m in (1, 31, 32, 1000, 8192):
        for w in (1, 2, 3, 8):
            blocks = shard.row_blocks(m, w)
            assert blocks[0][0] == 0 and blocks[-1][1] == m
            for (r0, r1), (s0, _) in zip(blocks, blocks[1:]):
                assert r1 == s0 and (r0 % 32 == 0 or r0 == r1 == m)
    assert shard.width_from_stats(0, 0) == (1, 0)
    assert shard.width_from_stats(5, 1) == (6, 1)
