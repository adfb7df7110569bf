"""Batched BiCGK / GESUMMV in one persistent launch, against the FP64 oracle.

Instances have log-uniform sizes (plus degenerate ones), are packed into
one buffer with per-instance offsets, either back to back (lda = n, rows
generally unaligned) or with rows padded to a multiple of 4 floats, and
are checked one by one.  A batched instance equals the same instance
batched alone bit for bit (fixed per-instance reduction order), and a
CUDA-graph replay gives the same bits as the direct launch.
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import built, dev, host  # noqa: F401
from tolerance import check_reduce

pytestmark = pytest.mark.gpu


def make_batch(kind, count, lo, hi, seed=0, extra=(), aligned=False):
    ms = synth.log_uniform_int(lo, hi, seed, synth.TID["sizes"], count).tolist()
    ns = synth.log_uniform_int(lo, hi, seed + 1, synth.TID["sizes"], count).tolist()
    shapes = list(zip(ms, ns)) + list(extra)
    # pack: matrices back to back (lda = n, so rows are generally unaligned),
    # or with rows padded to a multiple of 4 floats (every row 16-byte aligned)
    ldas = [(n + 3) // 4 * 4 if aligned else n for m, n in shapes]
    offs, total = [], 0
    for (m, n), ld in zip(shapes, ldas):
        offs.append(total)
        total += m * ld
    A = synth.uniform((max(total, 1),), seed, synth.TID["A"], device=dev())
    B = synth.uniform((max(total, 1),), seed, synth.TID["B"], device=dev()) if kind == "gesummv" else None
    descs, vecs = [], []
    for i, (m, n) in enumerate(shapes):
        x = synth.uniform((n,), seed + i, synth.TID["x"], device=dev())
        r = synth.uniform((m,), seed + i, synth.TID["r"], device=dev())
        y = torch.full((m,), float("nan"), device=dev())
        s = torch.full((n,), float("nan"), device=dev())
        d = {"m": m, "n": n, "lda": ldas[i], "A": A.data_ptr() + 4 * offs[i], "x": x, "r": r, "y": y, "s": s,
             "alpha": 1.5, "beta": 1.2}
        if B is not None:
            d["B"] = B.data_ptr() + 4 * offs[i]
        descs.append(d)
        vecs.append((x, r, y, s))
    return shapes, offs, A, B, descs, vecs


def run(kf, kind, descs, band_rows=0):
    seq = kf.KF_SEQ_BICGK if kind == "bicgk" else kf.KF_SEQ_GESUMMV
    b = kf.Batched(seq, descs, band_rows)
    ws = torch.zeros(b.workspace_size(), dtype=torch.uint8, device=dev())
    b.upload(ws)
    b.launch(ws)
    torch.cuda.synchronize()
    return b, ws


@pytest.mark.parametrize("aligned", [False, True])
@pytest.mark.parametrize("kind", ["bicgk", "gesummv"])
@pytest.mark.parametrize("band_rows", [32, 128])
def test_batched_parity(built, kind, band_rows, aligned):
    kf = built
    shapes, offs, A, B, descs, vecs = make_batch(kind, 40, 8, 700, seed=band_rows,
                                                 extra=[(1, 1), (1, 1500), (1500, 1), (2048, 1025), (33, 2049)],
                                                 aligned=aligned)
    run(kf, kind, descs, band_rows)
    Ah = A.cpu().numpy().astype(np.float64)
    Bh = B.cpu().numpy().astype(np.float64) if B is not None else None
    for (m, n), off, d, (x, r, y, s) in zip(shapes, offs, descs, vecs):
        ld = d["lda"]
        Am = Ah[off:off + m * ld].reshape(m, ld)[:, :n]
        xh, rh = host(x), host(r)
        if kind == "bicgk":
            qo, so = oracle.bicgk(Am, xh, rh)
            check_reduce(host(y), qo, oracle.abs_gemv(Am, xh), n, f"q {m}x{n}")
            check_reduce(host(s), so, oracle.abs_gemvt(Am, rh), m, f"s {m}x{n}")
        else:
            Bm = Bh[off:off + m * ld].reshape(m, ld)[:, :n]
            yo = oracle.gesummv(Am, Bm, xh, 1.5, 1.2)
            sc = 1.5 * oracle.abs_gemv(Am, xh) + 1.2 * oracle.abs_gemv(Bm, xh)
            check_reduce(host(y), yo, sc, n, f"y {m}x{n}")


@pytest.mark.parametrize("aligned", [False, True])
@pytest.mark.parametrize("kind", ["bicgk", "gesummv"])
def test_batched_instance_alone_bitwise_and_graph(built, kind, aligned):
    kf = built
    shapes, offs, A, B, descs, vecs = make_batch(kind, 64, 32, 2048, seed=7, aligned=aligned)
    b, ws = run(kf, kind, descs)
    ref = [(v[2].clone(), v[3].clone()) for v in vecs]
    for k in (0, 17, 63):
        alone = dict(descs[k])
        y2 = torch.empty_like(vecs[k][2]); s2 = torch.empty_like(vecs[k][3])
        alone["y"], alone["s"] = y2, s2
        run(kf, kind, [alone])
        assert torch.equal(y2, ref[k][0])
        if kind == "bicgk":
            assert torch.equal(s2, ref[k][1])
    # graph replay: same bits, twice (the queue and counters reset themselves)
    for v in vecs:
        v[2].fill_(float("nan")); v[3].fill_(float("nan"))
    b.capture(ws)
    for _ in range(2):
        b.replay()
        torch.cuda.synchronize()
        for (x, r, y, s), (y0, s0) in zip(vecs, ref):
            assert torch.equal(y, y0)
            if kind == "bicgk":
                assert torch.equal(s, s0)


def test_batched_empty_and_errors(built):
    kf = built
    b = kf.Batched(kf.KF_SEQ_BICGK, [])
    ws = torch.zeros(max(b.workspace_size(), 256), dtype=torch.uint8, device=dev())
    b.upload(ws)
    b.launch(ws)
    with pytest.raises(kf.KFError):
        kf.Batched(kf.KF_SEQ_ATAX, [])
    with pytest.raises(kf.KFError):
        kf.Batched(kf.KF_SEQ_BICGK, [{"m": 4, "n": 4, "lda": 2, "A": 256, "x": 256, "r": 256, "y": 256, "s": 256}])
