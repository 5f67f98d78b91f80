"""The row-sharded design of the dose and gradient evaluation, checked on the
host with two gloo ranks (CPU, 127.0.0.1) standing in for two GPUs; not
measured on hardware (every GPU machine of this project holds one GPU, and the
bench runs independent replicas).

Design: the rows are cut into one contiguous block per rank with equal entry
counts; rank k computes its rows' doses and its block's objective f_k and
gradient g_k = A_k^T r_k (here with the FP64 oracle); x is the same on every
rank.  The only exchange is f and g: every rank gathers all ranks' parts (a
gather moves bytes and adds nothing) and adds them in rank order, so every
rank holds the same bits and the result does not depend on which rank
finishes first (the reproducibility rule of Sec. II-D).  Checked: the ranks
agree bitwise; the result equals the same partition summed in one process
bitwise; doses equal the unsharded oracle bitwise (rows are independent); f and
g equal the unsharded oracle to FP64 rounding."""
import os
import socket

import numpy as np
import torch
import torch.distributed as td
import torch.multiprocessing as mp

import bench
import dosegen
import oracle

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    csr = dosegen.generate(dosegen.TINY)
    enc = oracle.encode(csr, oracle.U16_SCALE)
    p, w = dosegen.ellipsoid_target(dosegen.TINY)
    x = dosegen.spot_weights(csr.ncols, dosegen.weight_seed(dosegen.TINY))
    return csr, enc, x, p, w


def _block_result(block, ncols, x):
    nr, rp, col, a, p, w = block
    d = oracle.spmv(nr, rp, col, a, x)
    f, g = oracle.fgrad(nr, ncols, rp, col, a, x, p, w)
    return d, f, g


def _add_in_rank_order(fs, gs):
    f, g = fs[0], gs[0].copy()
    for fk, gk in zip(fs[1:], gs[1:]):
        f = f + fk
        g = g + gk
    return f, g


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        csr, enc, x, p, w = _problem()
        blocks = bench.oracle_row_blocks(enc.row_ptr, enc.col, enc.decoded, p, w, world)
        d, f, g = _block_result(blocks[rank], csr.ncols, x)
        fs = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        gs = [torch.zeros(csr.ncols, dtype=torch.float64) for _ in range(world)]
        td.all_gather(fs, torch.tensor([f], dtype=torch.float64))
        td.all_gather(gs, torch.from_numpy(g))
        f_all, g_all = _add_in_rank_order([float(t.item()) for t in fs], [t.numpy() for t in gs])
        q.put((rank, blocks[rank][0], d, f_all, g_all))
    finally:
        td.destroy_process_group()


def test_two_ranks_row_blocks_reduce_in_rank_order():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for pr in procs:
        pr.start()
    got = sorted((q.get(timeout=300) for _ in range(WORLD)), key=lambda t: t[0])
    for pr in procs:
        pr.join(120)
        assert pr.exitcode == 0
    csr, enc, x, p, w = _problem()
    # the partition: contiguous, covering, entry counts within one row of equal
    blocks = bench.oracle_row_blocks(enc.row_ptr, enc.col, enc.decoded, p, w, WORLD)
    assert sum(b[0] for b in blocks) == csr.nrows
    nnz_k = [int(b[1][-1]) for b in blocks]
    assert sum(nnz_k) == csr.nnz and abs(nnz_k[0] - nnz_k[1]) <= int(np.diff(enc.row_ptr.astype(np.int64)).max())
    # every rank holds the same bits
    for _, _, _, f_k, g_k in got[1:]:
        assert f_k == got[0][3] and np.array_equal(g_k.view(np.uint64), got[0][4].view(np.uint64))
    # the same partition summed in one process: bitwise
    parts = [_block_result(b, csr.ncols, x) for b in blocks]
    f_one, g_one = _add_in_rank_order([t[1] for t in parts], [t[2] for t in parts])
    assert got[0][3] == f_one and np.array_equal(got[0][4].view(np.uint64), g_one.view(np.uint64))
    # doses: the ranks' row blocks concatenated equal the unsharded oracle bitwise
    d_all = np.concatenate([t[2] for t in got])
    d_ref = oracle.spmv(csr.nrows, enc.row_ptr, enc.col, enc.decoded, x)
    assert np.array_equal(d_all.view(np.uint64), d_ref.view(np.uint64))
    # f and g: the unsharded oracle up to FP64 rounding of the regrouped sums
    f_ref, g_ref = oracle.fgrad(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, x, p, w)
    assert abs(got[0][3] - f_ref) <= 1e-12 * abs(f_ref)
    _, r = oracle.objective(d_ref, p, w)
    gabs = oracle.abs_spmv_t(csr.nrows, csr.ncols, enc.row_ptr, enc.col, enc.decoded, r)
    assert np.all(np.abs(got[0][4] - g_ref) <= 1e-12 * gabs + 1e-300)
