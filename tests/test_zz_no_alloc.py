"""The allocation-free entry point pic_sort_keys_noalloc.

It exists for callers that cannot call cudaMalloc (code whose device memory is
owned by another allocator, latency-critical loops where an allocation would
synchronise the device); its scratch is a fixed array inside the library.
Checked through the C ABI against the regroup that pic_load_particles already
performs with the same sort, on two calls in a row.  Kept in its own file so
that pytest runs it after every other test.
"""
import numpy as np
import pytest

from paper_1308_2590_gb300 import pic, workloads as W

pytestmark = pytest.mark.gpu


def _case(seed, tile, n_cells=(48, 40), ppc=24):
    cfg = W.uniform_plasma("noalloc", n_cells[0], ppc, 1, seed=seed, tile=tile)
    cfg.ny = n_cells[1]
    cfg.species = cfg.species[:1]
    P = W.generate_particles(cfg)[0]
    # tile key exactly as the library forms it after a load: 2 * tile id of the cell
    cx = np.floor(P["x"] / cfg.dx).astype(np.int64)
    cy = np.floor(P["y"] / cfg.dy).astype(np.int64)
    ntx = -(-cfg.nx // tile)
    nty = -(-cfg.ny // tile)
    keys = (2 * ((cy // tile) * ntx + cx // tile)).astype(np.uint32)
    return cfg, P, keys, 2 * ntx * nty + 2


def _expected_order(cfg, P, stream):
    """The existing entry point: pic_load_particles regroups the species stably by tile."""
    with pic.Pic(cfg, stream=stream) as g:
        g.load(0, P)
        return g.pic_get_particles(0)


def test_noalloc_sort_matches_existing_regroup_twice_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    stream = torch.cuda.current_stream().cuda_stream
    cases = [_case(seed=2024, tile=8), _case(seed=2025, tile=4, n_cells=(64, 37), ppc=40)]
    expected = [_expected_order(cfg, P, stream) for (cfg, P, _, _) in cases]
    perms = []
    for (cfg, P, keys, max_key) in cases:          # two calls in a row
        kd = torch.from_numpy(keys.view(np.int32)).cuda()
        pd = torch.full((keys.size,), -1, dtype=torch.int32, device="cuda")
        pic.pic_sort_keys_noalloc(kd.data_ptr(), keys.size, max_key, pd.data_ptr(), stream)
        perms.append((kd, pd))
    torch.cuda.synchronize()
    for (cfg, P, keys, _), exp, (_, pd) in zip(cases, expected, perms):
        perm = pd.cpu().numpy().astype(np.int64)
        assert np.array_equal(np.sort(perm), np.arange(keys.size))             # a permutation
        assert np.all(np.diff(keys[perm].astype(np.int64)) >= 0)                 # sorted
        Lx, Ly = cfg.nx * cfg.dx, cfg.ny * cfg.dy
        # same order as the library's regroup, within the parity tolerance (1e-10 relative)
        assert np.max(np.abs(P["x"][perm] - exp["x"])) <= 1e-10 * Lx
        assert np.max(np.abs(P["y"][perm] - exp["y"])) <= 1e-10 * Ly
        for k in ("ux", "uy", "uz", "w"):
            scale = np.max(np.abs(P[k])) + 1e-300
            assert np.max(np.abs(P[k][perm] - exp[k])) <= 1e-10 * scale


def test_noalloc_sort_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    kd = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(pic.PicError, match="PIC_ERR_CAPACITY"):
        pic.pic_sort_keys_noalloc(kd.data_ptr(), pic.NOALLOC_MAX_KEYS + 1, 10, kd.data_ptr(), None)


def test_noalloc_sort_three_passes_against_a_stable_argsort():
    """Keys up to 2^20 (three 8-bit passes, ping-pong through both scratch buffers) against numpy's
    stable argsort of the same keys."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    rng = np.random.default_rng(31)
    keys = rng.integers(0, 1 << 20, size=300_001).astype(np.uint32)
    keys[::7] = keys[3]                                  # many equal keys: stability matters
    kd = torch.from_numpy(keys.view(np.int32)).cuda()
    pd = torch.full((keys.size,), -1, dtype=torch.int32, device="cuda")
    pic.pic_sort_keys_noalloc(kd.data_ptr(), keys.size, int(keys.max()), pd.data_ptr(), None)
    torch.cuda.synchronize()
    assert np.array_equal(pd.cpu().numpy().astype(np.int64), np.argsort(keys, kind="stable"))
