"""Loads of several species in one call (pic_load_species) on the GPU.

The call must leave bitwise the same state as pic_load_particles species by
species (into empty species, where one species' regroup overlaps the next
species' conversion, and into species that already hold particles), from
page-locked and pageable host arrays and from device arrays; and it is all
or nothing: an invalid particle in any species loads nothing.  A prefetched
load (pic_prefetch_species, then pic_load_prefetched) must leave the state
the direct load leaves, with up to two loads prefetched ahead.
"""
import numpy as np
import pytest

from paper_1308_2590_gb300 import pic, workloads as W
from tests.parity import stream
from tests.test_gpu_parity import hot, small_foil, small_uniform

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "ux", "uy", "uz", "w")


def _state(g, nsp):
    out = [g.pic_moments(), *g.pic_fields()]
    for s in range(nsp):
        P = g.pic_get_particles(s)
        out += [P[k] for k in KEYS + ("cell",)]
    return out


def _equal(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x.shape == y.shape and np.array_equal(x.view(np.uint8), y.view(np.uint8))


def _pinned(parts):
    torch = pytest.importorskip("torch")
    return [{k: torch.from_numpy(np.ascontiguousarray(P[k])).pin_memory().numpy() for k in KEYS} for P in parts]


def _cfgs():
    a = small_foil()
    b = hot(small_uniform(tile=4), 20.0)
    c = small_foil(precision=W.PREC_FP32)
    for cfg in (a, b, c):
        cfg.deposit = W.DEPOSIT_DETERMINISTIC
    return [a, b, c]


@pytest.mark.parametrize("k", [0, 1, 2])
@pytest.mark.parametrize("memory", ["pinned", "pageable"])
def test_load_species_equals_per_species_loads(k, memory):
    cfg = _cfgs()[k]
    parts = W.generate_particles(cfg)
    src = _pinned(parts) if memory == "pinned" else parts
    ref = pic.Pic(cfg, stream=stream())
    for s, P in enumerate(src):
        ref.load(s, P)
    got = pic.Pic(cfg, stream=stream())
    got.pic_load_species(src)
    _equal(_state(ref, len(parts)), _state(got, len(parts)))
    ref.pic_step(4)
    got.pic_step(4)
    _equal(_state(ref, len(parts)), _state(got, len(parts)))
    # a second load into species that now hold particles (no overlap, checks first)
    more = W.generate_particles(cfg, seed=cfg.seed + 1)
    for s, P in enumerate(more):
        ref.load(s, P)
    got.pic_load_species(more)
    ref.pic_step(2)
    got.pic_step(2)
    _equal(_state(ref, len(parts)), _state(got, len(parts)))
    # after a clear the species are empty again: the overlapped path
    ref.pic_clear_particles()
    got.pic_clear_particles()
    for s, P in enumerate(src):
        ref.load(s, P)
    got.pic_load_species(src)
    ref.pic_step(1)
    got.pic_step(1)
    _equal(_state(ref, len(parts)), _state(got, len(parts)))
    ref.close()
    got.close()


def test_load_species_partial_and_empty_entries():
    cfg = _cfgs()[0]
    parts = W.generate_particles(cfg)
    ref = pic.Pic(cfg, stream=stream())
    ref.load(1, parts[1])
    got = pic.Pic(cfg, stream=stream())
    got.pic_load_species([{k: parts[0][k][:0] for k in KEYS}, parts[1]])
    _equal(_state(ref, 2), _state(got, 2))
    got.pic_load_species([parts[0]])          # fewer entries than species
    ref.load(0, parts[0])
    _equal(_state(ref, 2), _state(got, 2))
    got.pic_load_species([])
    _equal(_state(ref, 2), _state(got, 2))
    with pytest.raises(pic.PicError):
        got.pic_load_species(parts + [parts[0]])   # more entries than species
    ref.close()
    got.close()


@pytest.mark.parametrize("fresh", [True, False])
@pytest.mark.parametrize("memory", ["pinned", "pageable"])
def test_load_species_is_all_or_nothing(fresh, memory):
    cfg = _cfgs()[0]
    parts = W.generate_particles(cfg)
    g = pic.Pic(cfg, stream=stream())
    if not fresh:
        g.load(0, parts[0])
    before = _state(g, 2)
    counts = [g.pic_particle_count(s) for s in range(2)]
    bad = [{k: v.copy() for k, v in P.items()} for P in parts]
    bad[1]["x"][len(bad[1]["x"]) // 2] = cfg.nx * cfg.dx * 2.0      # outside the box
    src = _pinned(bad) if memory == "pinned" else bad
    with pytest.raises(pic.PicError, match="species 1"):
        g.pic_load_species(src)
    assert [g.pic_particle_count(s) for s in range(2)] == counts
    _equal(before, _state(g, 2))
    # a NaN velocity is refused the same way
    bad = [{k: v.copy() for k, v in P.items()} for P in parts]
    bad[0]["uz"][3] = np.nan
    with pytest.raises(pic.PicError, match="species 0"):
        g.pic_load_species(_pinned(bad) if memory == "pinned" else bad)
    _equal(before, _state(g, 2))
    # and the handle still works: a valid load and steps equal a clean run
    g.pic_load_species(parts if fresh else [{k: parts[0][k][:0] for k in KEYS}, parts[1]])
    g.pic_step(3)
    ref = pic.Pic(cfg, stream=stream())
    for s, P in enumerate(parts):
        ref.load(s, P)
    ref.pic_step(3)
    _equal(_state(ref, 2), _state(g, 2))
    ref.close()
    g.close()


def test_load_species_from_device_arrays():
    """Arrays in device memory (CUDA tensors) give bitwise the state of host arrays."""
    import ctypes
    torch = pytest.importorskip("torch")
    cfg = _cfgs()[0]
    parts = W.generate_particles(cfg)
    ref = pic.Pic(cfg, stream=stream())
    ref.pic_load_species(parts)
    dev = [{k: torch.from_numpy(np.ascontiguousarray(P[k])).cuda() for k in KEYS} for P in parts]
    torch.cuda.synchronize()
    sd = (pic.PicSpeciesData * len(dev))()
    for s, P in enumerate(dev):
        sd[s].n = P["x"].numel()
        sd[s].x, sd[s].y, sd[s].ux, sd[s].uy, sd[s].uz, sd[s].w = [ctypes.c_void_p(P[k].data_ptr()) for k in KEYS]
    got = pic.Pic(cfg, stream=stream())
    # an invalid particle in device memory is refused (and reported) first
    dev[1]["x"][5] = cfg.nx * cfg.dx * 3.0
    torch.cuda.synchronize()
    assert pic.lib().pic_load_species(got.h, len(dev), sd) == pic.PIC_ERR_ARG
    assert b"species 1 particle 5" in pic.lib().pic_last_error()
    assert [got.pic_particle_count(s) for s in range(2)] == [0, 0]
    dev[1]["x"][5] = float(parts[1]["x"][5])
    torch.cuda.synchronize()
    assert pic.lib().pic_load_species(got.h, len(dev), sd) == 0, pic.lib().pic_last_error()
    _equal(_state(ref, 2), _state(got, 2))
    ref.pic_step(3)
    got.pic_step(3)
    _equal(_state(ref, 2), _state(got, 2))
    ref.close()
    got.close()


@pytest.mark.parametrize("k,memory", [(0, "pinned"), (1, "pinned"), (2, "pinned"), (0, "pageable")])
def test_prefetched_loads_equal_direct_loads(k, memory):
    cfg = _cfgs()[k]
    first = W.generate_particles(cfg)
    second = W.generate_particles(cfg, seed=cfg.seed + 1)
    if memory == "pinned":
        first, second = _pinned(first), _pinned(second)
    ref = pic.Pic(cfg, stream=stream())
    got = pic.Pic(cfg, stream=stream())
    ref.pic_load_species(first)
    got.pic_prefetch_species(first)
    got.pic_prefetch_species(second)           # two loads wait
    with pytest.raises(pic.PicError):
        got.pic_prefetch_species(first)        # a third is refused
    got.pic_load_prefetched()
    _equal(_state(ref, len(first)), _state(got, len(first)))
    ref.pic_step(3)
    got.pic_step(3)
    ref.pic_clear_particles()
    got.pic_clear_particles()
    ref.pic_load_species(second)
    got.pic_load_prefetched()                  # copied while the steps ran
    got.pic_prefetch_species(first)            # the freed slot takes the next one
    ref.pic_step(2)
    got.pic_step(2)
    _equal(_state(ref, len(first)), _state(got, len(first)))
    ref.pic_load_species(first)                # into species that hold particles
    got.pic_load_prefetched()
    ref.pic_step(1)
    got.pic_step(1)
    _equal(_state(ref, len(first)), _state(got, len(first)))
    with pytest.raises(pic.PicError):
        got.pic_load_prefetched()              # nothing left
    ref.close()
    got.close()


def test_prefetched_load_with_an_invalid_particle_loads_nothing():
    cfg = _cfgs()[0]
    parts = _pinned(W.generate_particles(cfg))
    bad = [{k: v.copy() for k, v in P.items()} for P in parts]
    bad[1]["x"][7] = cfg.nx * cfg.dx * 2.0     # outside the box
    g = pic.Pic(cfg, stream=stream())
    g.pic_prefetch_species(_pinned(bad))
    g.pic_prefetch_species(parts)
    with pytest.raises(pic.PicError, match="species 1 particle 7"):
        g.pic_load_prefetched()
    assert [g.pic_particle_count(s) for s in range(2)] == [0, 0]
    g.pic_load_prefetched()                    # the next prefetched load is intact
    ref = pic.Pic(cfg, stream=stream())
    ref.pic_load_species(parts)
    _equal(_state(ref, len(parts)), _state(g, len(parts)))
    g.close()
    ref.close()
