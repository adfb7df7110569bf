"""Host-side tables of the library, without a GPU.

The batched form builds its instance descriptors and tile list on the host
(kf_batched_create records device pointers and never reads them), and the
tuning cache is a host map with a text file format.  Both run here; the
launches that use them are in the GPU tests.
"""

import ctypes

import pytest

import synth

FAKE = 1 << 20      # stand-in device address: creation only records pointers


@pytest.fixture(scope="module")
def kf():
    from paper_1305_1183_gb300 import _build, kf as K
    _build.build()
    K.lib()
    return K


def _descs(sizes, gesummv=False):
    return [dict(m=m, n=n, lda=n, A=FAKE, B=FAKE if gesummv else None, x=FAKE, r=None if gesummv else FAKE,
                 y=FAKE, s=None if gesummv else FAKE, alpha=1.5, beta=1.2) for m, n in sizes]


def _sizes(count, seed=0):
    m = synth.log_uniform_int(32, 2048, seed, synth.TID["sizes"], count).tolist()
    n = synth.log_uniform_int(32, 2048, seed + 1, synth.TID["sizes"], count).tolist()
    return list(zip(m, n))


def test_batched_bytes_follow_the_byte_model(kf):
    """One launch moves each matrix once and each vector once:
    BiCGK 4mn + 8(m + n), GESUMMV 8mn + 4(m + n) bytes per instance."""
    sizes = _sizes(300)
    _, b = kf.Batched(kf.KF_SEQ_BICGK, _descs(sizes)).info()
    assert b == sum(4 * m * n + 8 * (m + n) for m, n in sizes)
    _, b = kf.Batched(kf.KF_SEQ_GESUMMV, _descs(sizes, gesummv=True)).info()
    assert b == sum(8 * m * n + 4 * (m + n) for m, n in sizes)


def test_batched_tiles_cover_every_band(kf):
    """Every instance has at least one tile per band of rows; a lower band
    height never gives fewer tiles; a tiny instance is one tile."""
    sizes = _sizes(200, seed=3)
    prev = None
    for band in (512, 256, 128, 64, 32):
        t, _ = kf.Batched(kf.KF_SEQ_BICGK, _descs(sizes), band_rows=band).info()
        assert t >= sum(-(-m // band) for m, _ in sizes)
        if prev is not None:
            assert t >= prev
        prev = t
    assert kf.Batched(kf.KF_SEQ_BICGK, _descs([(32, 100)]), band_rows=32).info()[0] == 1
    assert kf.Batched(kf.KF_SEQ_BICGK, _descs([]), band_rows=32).info() == (0, 0.0)


def test_batched_workspace_bound_covers_every_band(kf):
    sizes = _sizes(100, seed=5)
    arr = kf._desc_array(_descs(sizes))
    bound = ctypes.c_size_t(0)
    assert kf.lib().kf_batched_workspace_bound(kf.KF_SEQ_BICGK, ctypes.cast(arr, ctypes.c_void_p), len(sizes),
                                               ctypes.byref(bound)) == 0
    sizes_ws = [kf.Batched(kf.KF_SEQ_BICGK, _descs(sizes), band_rows=b).workspace_size()
                for b in (32, 64, 128, 256, 512)]
    assert max(sizes_ws) <= bound.value
    # row partials alone need 4 bytes per row of every instance
    assert min(sizes_ws) >= 4 * sum(m for m, _ in sizes)
    small = kf.Batched(kf.KF_SEQ_BICGK, _descs(sizes[:10])).workspace_size()
    assert small < kf.Batched(kf.KF_SEQ_BICGK, _descs(sizes)).workspace_size()


def test_batched_rejects_bad_requests(kf):
    L = kf.lib()

    def create(seq, descs, band=0):
        arr = kf._desc_array(descs)
        h = ctypes.c_void_p()
        st = L.kf_batched_create(seq, ctypes.cast(arr, ctypes.c_void_p), len(descs), band, ctypes.byref(h))
        if st == 0:
            L.kf_batched_destroy(h)
        return st

    good = _descs([(64, 64)] * 4)
    assert create(kf.KF_SEQ_BICGK, good) == 0
    assert create(kf.KF_SEQ_BICGK, good, band=48) == kf.KF_ERR_INVALID_ARG      # not a multiple of 32
    assert create(kf.KF_SEQ_BICGK, good, band=8192) == kf.KF_ERR_INVALID_ARG
    assert create(kf.KF_SEQ_GEMVER, good) == kf.KF_ERR_UNSUPPORTED
    bad = _descs([(64, 64)] * 4)
    bad[3]["lda"] = 32                                                           # lda < n
    assert create(kf.KF_SEQ_BICGK, bad) == kf.KF_ERR_INVALID_ARG
    assert b"instance 3" in L.kf_last_error()
    bad = _descs([(64, 64)] * 2, gesummv=True)
    bad[1]["B"] = None                                                           # GESUMMV needs B
    assert create(kf.KF_SEQ_GESUMMV, bad) == kf.KF_ERR_INVALID_ARG
    bad = _descs([(64, 64)])
    bad[0]["s"] = None                                                           # BiCGK needs s
    assert create(kf.KF_SEQ_BICGK, bad) == kf.KF_ERR_INVALID_ARG
    empty = _descs([(0, 64), (64, 0)])
    empty[0].update(A=None, r=None, y=None)
    empty[1].update(A=None, x=None, s=None)
    assert create(kf.KF_SEQ_BICGK, empty) == 0                                   # empty instances need no pointers


def test_tuning_cache_file_round_trip(kf, tmp_path):
    """Entries load only under the device line the library writes for this
    device; a saved cache holds what was loaded; malformed lines fail."""
    L = kf.lib()
    n = ctypes.c_int(0)
    kf.kf_tune_cache_clear()
    try:
        p0 = tmp_path / "empty.txt"
        assert L.kf_tune_cache_save(str(p0).encode()) == 0
        lines = p0.read_text().splitlines()
        assert lines[0].startswith("#")
        dev = [ln for ln in lines if ln.startswith("device ")]
        assert len(dev) == 1 and len(lines) == 2
        f = tmp_path / "cache.txt"
        f.write_text(f"# hand-written\n{dev[0]}\nmat key one : 8 2 2 0 4\nvec key two : 256 4 1\n"
                     "atax 13 13 : 1 1 1 0 0\ngemver_form 13 : 1 0 0 0 0\nsgemvt_form 12 13 : 2 0 0 0 0\n"
                     "device another_part_sm1\nmat foreign : 8 1 4 0 4\n")
        assert L.kf_tune_cache_load(str(f).encode(), ctypes.byref(n)) == 0
        assert n.value == 5
        assert L.kf_tune_cache_entries(ctypes.byref(n)) == 0 and n.value == 5
        p1 = tmp_path / "saved.txt"
        assert L.kf_tune_cache_save(str(p1).encode()) == 0
        saved = p1.read_text().splitlines()
        assert "mat key one : 8 2 2 0 4" in saved and "vec key two : 256 4 1" in saved
        assert "atax 13 13 : 1 1 1 0 0" in saved and "gemver_form 13 : 1 0 0 0 0" in saved
        assert "sgemvt_form 12 13 : 2 0 0 0 0" in saved
        assert not any("foreign" in ln for ln in saved)
        g = tmp_path / "broken.txt"
        g.write_text(f"{dev[0]}\nmat no separator 8 2 2 0 4\n")
        assert L.kf_tune_cache_load(str(g).encode(), ctypes.byref(n)) == kf.KF_ERR_INVALID_ARG
        assert b"malformed" in L.kf_last_error()
        assert L.kf_tune_cache_load(str(tmp_path / "missing.txt").encode(), ctypes.byref(n)) == kf.KF_ERR_INVALID_ARG
    finally:
        kf.kf_tune_cache_clear()
