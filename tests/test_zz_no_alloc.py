"""pic_op_sort_noalloc (the by-cell compaction with its scratch in a static
__device__ array) against the context's own compaction, pic_compact.

Sorting is integer work, so every kept particle's record must match bit for
bit; the order of particles inside one cell is unspecified on both sides, so
the comparison is per id, plus the per-cell counts and the cell order of the
output.  Two calls in a row check that the shared scratch is cleared between
calls.  Collected last so that it also runs after every other GPU test.
"""
import numpy as np
import pytest

from paper_1607_04069_gb300 import workloads as W

from helpers import gpu_discharge

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def _input(n, n_cells, p64, seed):
    """n slots, about 1 in 7 removed, positions over the whole gap."""
    rng = np.random.default_rng(seed)
    xi = rng.uniform(0.0, n_cells, n)
    dead = rng.random(n) < 1.0 / 7.0
    if p64:
        pos = np.where(dead, -1.0, xi)
    else:
        pos = rng.integers(1, 2**32, n, dtype=np.uint64).astype(np.uint32)
        pos[dead] = 0
    v = [rng.normal(0.0, 1e5, n).astype(np.float32) for _ in range(3)]
    ids = rng.permutation(np.arange(1, n + 1, dtype=np.uint64)) | np.uint64(5 << 40)
    return pos, v, ids


def _xi(pos, n_cells, p64):
    return pos.astype(np.float64) if p64 else pos.astype(np.float64) * (n_cells / 2.0**32)


def _run_noalloc(torch, pos, v, ids, n_cells, p64):
    import paper_1607_04069_gb300 as P
    n = pos.size
    dev = torch.device("cuda", 0)
    tp = torch.from_numpy(pos.copy() if p64 else pos.view(np.int32).copy()).to(dev)   # float64 selects 64-bit
    tv = [torch.from_numpy(a.copy()).to(dev) for a in v]
    tid = torch.from_numpy(ids.view(np.int64).copy()).to(dev)
    outs = [torch.full((n,), -7, dtype=t.dtype, device=dev) for t in (tp, *tv, tid)]
    n_out = torch.full((1,), -1, dtype=torch.int64, device=dev)
    P.op_sort_noalloc(tp, *tv, tid, n_cells, *outs, n_out=n_out)
    torch.cuda.synchronize()
    m = int(n_out.item())
    host = [o[:m].cpu().numpy() for o in outs]
    return {"xi": _xi(host[0].view(np.float64 if p64 else np.uint32), n_cells, p64), "vx": host[1],
            "vy": host[2], "vz": host[3], "id": host[4].view(np.uint64)}


def _check_sorted_by_cell(r, n_cells):
    cell = np.floor(r["xi"]).astype(np.int64)
    assert np.all(np.diff(cell) >= 0), "output not in cell order"
    return np.bincount(cell, minlength=n_cells)


def _same_records(a, b):
    oa, ob = np.argsort(a["id"]), np.argsort(b["id"])
    for k in ("id", "xi", "vx", "vy", "vz"):
        assert np.array_equal(a[k][oa], b[k][ob]), k


@pytest.mark.parametrize("p64", [False, True], ids=["u32", "f64"])
def test_two_calls_match_pic_compact(torch, p64):
    cfg = W.ccp_small(n_per_species=20_000)
    cfg.update(pos_precision=64 if p64 else 32, sort_every_e=0, sort_every_i=0)
    n_cells = cfg["n_cells"]
    n = 20_003                                      # ragged: not a multiple of 4 or of a warp
    pos, v, ids = _input(n, n_cells, p64, seed=11)
    d = gpu_discharge(cfg)
    d.set_species(0, pos, *v, ids)
    d.compact(0)
    ref = d.get_species(0)
    d.close()
    ref_counts = _check_sorted_by_cell(ref, n_cells)
    alive = (pos >= 0.0) if p64 else (pos != 0)
    assert len(ref["id"]) == int(alive.sum())
    for _ in range(2):                              # the second call reuses the static scratch
        got = _run_noalloc(torch, pos, v, ids, n_cells, p64)
        assert len(got["id"]) == len(ref["id"])
        assert np.array_equal(_check_sorted_by_cell(got, n_cells), ref_counts)
        _same_records(got, ref)


def test_max_cells_and_empty(torch):
    """n_cells at the scratch limit (4096) against per-cell counts taken on the
    host, then an empty input, which must report zero kept."""
    n_cells, n = 4096, 300_001
    pos, v, ids = _input(n, n_cells, False, seed=12)
    got = _run_noalloc(torch, pos, v, ids, n_cells, False)
    live = pos != 0
    counts = np.bincount((pos[live] >> np.uint32(20)).astype(np.int64), minlength=n_cells)
    assert np.array_equal(_check_sorted_by_cell(got, n_cells), counts)
    want = {"xi": _xi(pos[live], n_cells, False), "vx": v[0][live], "vy": v[1][live], "vz": v[2][live],
            "id": ids[live]}
    _same_records(got, want)
    empty = _run_noalloc(torch, pos[:0], [a[:0] for a in v], ids[:0], n_cells, False)
    assert len(empty["id"]) == 0


def test_rejects_cells_above_scratch(torch):
    import paper_1607_04069_gb300 as P
    dev = torch.device("cuda", 0)
    a = torch.zeros(8, dtype=torch.int32, device=dev)
    f = torch.zeros(8, dtype=torch.float32, device=dev)
    i = torch.zeros(8, dtype=torch.int64, device=dev)
    with pytest.raises(P.PicError) as e:
        P.op_sort_noalloc(a, f, f, f, i, 8192, a.clone(), f.clone(), f.clone(), f.clone(), i.clone())
    assert "4096" in str(e.value)
