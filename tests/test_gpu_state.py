"""Checkpoint / resume (pic_get_state, pic_set_state) and immobile species.

* A run that is checkpointed after 5 steps and resumed in a fresh context
  follows the uninterrupted run: fields, current, particles (by id) and
  energies within 1e-12 after 6 more steps (the only difference is the
  summation order of the floating-point atomics), FP64 and mixed, with the
  binned store and the sort phase restored.
* set_state refuses a blob of another grid descriptor, a truncated blob and
  a foreign byte string, and leaves the context usable.
* An immobile species is stored as nothing and changes nothing: a run with
  electrons plus an immobile background equals the electron-only run.
* A species that grows beyond its store (re-allocation) uploads whole, from
  pinned or pageable host arrays.
* Right after a load (its sort leaves the record moves to the next particle
  step), reading the particles, counting them, the kinetic energy, a
  checkpoint and the tape all see the loaded particles.
"""
import numpy as np
import pytest

from paper_1608_01009_gb300 import pic as P
from paper_1608_01009_gb300 import workloads as W
from tests import parity as PT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _two_species():
    wl = W.uniform_plasma((16, 8, 12), 6, 0.05, 0.2, seed=61)
    pos = W.uniform_plasma((16, 8, 12), 3, 0.05, 0.1, seed=62, q=1.0, m=1.0)
    wl.species = wl.species + pos.species
    return wl


def _snapshot(sim, nspecies):
    E, B = sim.get_fields()
    J = sim.get_current()
    parts = []
    for s in range(nspecies):
        p = sim.get_particles(s)
        o = np.argsort(p["id"])
        parts.append({k: v[o] for k, v in p.items()})
    return E, B, J, parts, sim.energy()


def _compare(a, b, tol):
    for x, y in zip(a[:3], b[:3]):
        assert PT.rel_err(x, y) <= tol
    for pa, pb in zip(a[3], b[3]):
        assert np.array_equal(pa["id"], pb["id"])
        for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
            assert PT.rel_err(pa[k], pb[k]) <= tol, k
    for ea, eb in zip(a[4], b[4]):
        assert abs(ea - eb) <= tol * abs(eb)


@pytest.mark.parametrize("precision,tol", [(P.FP64, 1e-12), (P.MIXED, 1e-6)])
def test_checkpoint_resume_follows_the_uninterrupted_run(precision, tol):
    wl = _two_species()
    a = PT.make_sim(wl, precision=precision)
    a.step(5)
    blob = a.get_state()
    a.step(6)
    ref = _snapshot(a, 2)
    b = PT.make_sim(W.uniform_plasma((16, 8, 12), 1, 0.05, 0.0, seed=1), precision=precision)  # other particles
    b.set_state(blob)
    assert b.nspecies == 2
    assert b.species_info(1) == {"q": 1.0, "m": 1.0, "immobile": False, "nid": wl.species[1].n}
    b.step(6)
    _compare(_snapshot(b, 2), ref, tol)
    a.close()
    b.close()


def test_set_state_rejects_foreign_blobs_and_stays_usable():
    wl = W.config("c1")
    a = PT.make_sim(wl)
    a.step(2)
    blob = a.get_state()
    other = P.Simulation((16, 16, 8), wl.d, wl.dt)  # another grid
    with pytest.raises(P.PicError) as ei:
        other.set_state(blob)
    assert ei.value.code == -1
    other.close()
    with pytest.raises(P.PicError):
        a.set_state(blob[: len(blob) // 2])
    with pytest.raises(P.PicError):
        a.set_state(b"\0" * len(blob))
    # refused blobs leave the context as it was
    ref = _snapshot(a, 1)
    a.set_state(blob)
    _compare(_snapshot(a, 1), ref, 1e-14)  # energies are re-summed in another order
    a.step(1)
    a.sync()
    a.close()


def test_immobile_background_is_not_stored_and_changes_nothing():
    wl = W.config("c1")
    sp = wl.species[0]
    a = PT.make_sim(wl)
    b = PT.make_sim(wl)
    ion = b.add_species(1.0, 1836.0, *sp.arrays(), immobile=True)
    assert ion == 1 and b.count(ion) == 0
    assert b.species_info(ion)["immobile"]
    a.step(5)
    b.step(5)
    Ea, Ba = a.get_fields()
    Eb, Bb = b.get_fields()
    assert PT.rel_err(Eb, Ea) <= 1e-12 and PT.rel_err(Bb, Ba) <= 1e-12
    assert b.get_particles(ion)["x"].size == 0
    assert abs(b.energy()[1] - a.energy()[1]) <= 1e-12 * a.energy()[1]
    a.close()
    b.close()


def test_pinned_host_arrays_load_like_pageable_ones():
    # page-locked host arrays are read in place by the load kernel; pageable
    # ones are staged: the stored particles must be identical
    wl = W.config("c1")
    sp = wl.species[0]
    a = PT.make_sim(wl)
    b = PT.make_sim(wl)
    pinned = []
    for arr in sp.arrays():
        t = torch.empty(arr.shape[0], dtype=torch.float64, pin_memory=True)
        t.numpy()[:] = arr
        pinned.append(t)
    b.set_particles(0, *[t.numpy() for t in pinned])
    pa, pb = a.get_particles(0), b.get_particles(0)
    oa, ob = np.argsort(pa["id"]), np.argsort(pb["id"])
    for k in ("id", "x", "y", "z", "ux", "uy", "uz", "w"):
        assert np.array_equal(pa[k][oa], pb[k][ob]), k
    a.step(3)
    b.step(3)
    assert PT.rel_err(b.get_fields()[0], a.get_fields()[0]) <= 1e-13
    a.close()
    b.close()


def test_bounded_wait_times_out_and_the_context_recovers():
    # the particle kernel's bounded barrier wait, on a barrier nothing completes:
    # it gives up, the host reads PIC_ERR_TIMEOUT, the context keeps working
    wl = W.config("c1")
    sim = PT.make_sim(wl)
    sim.step(2)
    assert sim.selftest_wait_timeout() == -8  # PIC_ERR_TIMEOUT
    sim.step(2)
    sim.sync()
    wf, wk = sim.energy()
    assert np.isfinite(wf) and np.isfinite(wk)
    sim.close()


HEADER = 144  # state blob header bytes (the since_sort counter is its last 8)


def _cell_offset(wl):
    """Byte offset of species 0's packed cells in a state blob of the current format:
    header (120 B), padded E|B (6 P) and J (3 P) plus the folded current
    (3 cells) in doubles, then the 40-byte species record."""
    P = (wl.n[0] + 4) * (wl.n[1] + 4) * (wl.n[2] + 4)
    ncell = wl.n[0] * wl.n[1] * wl.n[2]
    return HEADER + (9 * P + 3 * ncell) * 8 + 40


def _pad8(x):
    return (x + 7) & ~7


def _chunk_table(blob, wl, n, nbins, real=8):
    """Offsets of species 0's bin starts and chunk table, and the chunk count
    (from the species record), in a state blob of the current format."""
    cells = _cell_offset(wl)
    nch = int(np.frombuffer(bytes(blob[cells - 4:cells]), dtype=np.int32)[0])
    bins = cells + 2 * _pad8(4 * n) + 7 * _pad8(real * n)
    return bins, bins + _pad8(4 * (nbins + 1)), nch


def test_set_state_bounds_every_chunk_and_the_sort_counter():
    # a chunk longer than CHUNK (the particle kernel's per-CTA queue slots), a
    # chunk that leaves its bin, and a since-sort counter beyond the sort
    # interval are refused before any kernel sees them
    wl = W.uniform_plasma((8, 8, 8), 100, 0.05, 0.05, seed=63)  # 6400 particles per 4^3 bin
    sim = PT.make_sim(wl)
    good = bytearray(sim.get_state())
    n, nbins = wl.nparticles, 8
    bins, chunks, nch = _chunk_table(good, wl, n, nbins)
    table = np.frombuffer(bytes(good[chunks:chunks + 16 * nch]), dtype=np.int32).reshape(nch, 4).copy()
    starts = np.frombuffer(bytes(good[bins:bins + 4 * (nbins + 1)]), dtype=np.int32)
    assert nch == 2 * nbins and table[0, 0] == table[1, 0] == 0  # bin 0 cut into two chunks
    assert table[0, 2] + table[1, 2] == starts[1] - starts[0] > 4096
    bad = bytearray(good)  # bin 0 as one chunk of 6400 particles
    t = table.copy()
    t[0, 2] = starts[1] - starts[0]
    bad[chunks:chunks + 16 * nch] = t.tobytes()
    with pytest.raises(P.PicError) as ei:
        sim.set_state(bytes(bad))
    assert ei.value.code == -1
    bad = bytearray(good)  # a chunk of bin 0 that runs into bin 1
    t = table.copy()
    t[1, 2] += 1
    bad[chunks:chunks + 16 * nch] = t.tobytes()
    with pytest.raises(P.PicError) as ei:
        sim.set_state(bytes(bad))
    assert ei.value.code == -1
    bad = bytearray(good)  # steps since the last sort beyond the sort interval
    bad[HEADER - 8:HEADER] = np.array([1000], dtype=np.int64).tobytes()
    with pytest.raises(P.PicError) as ei:
        sim.set_state(bytes(bad))
    assert ei.value.code == -1
    sim.set_state(bytes(good))  # the context is still usable
    sim.step(2)
    sim.sync()
    sim.close()


def test_particle_outside_its_supercell_slack_is_flagged():
    # a valid cell far from its chunk's supercell: the particle kernel's own
    # bounds check flags it (PIC_ERR_BIN_OVERFLOW) and touches no tile for it
    wl = W.config("c1")
    sim = PT.make_sim(wl)
    blob = bytearray(sim.get_state())
    off = _cell_offset(wl)
    far = np.array([9 | (9 << 10) | (9 << 20)], dtype=np.int32).tobytes()
    blob[off:off + 4] = far
    sim.set_state(bytes(blob))
    sim.step(1)
    with pytest.raises(P.PicError) as ei:
        sim.sync()
    assert ei.value.code == -4  # PIC_ERR_BIN_OVERFLOW
    sim.close()
    # a cell outside the grid never reaches a kernel: set_state refuses it
    sim = PT.make_sim(wl)
    blob = bytearray(sim.get_state())
    blob[off:off + 4] = np.array([40 | (1 << 10)], dtype=np.int32).tobytes()
    with pytest.raises(P.PicError) as ei:
        sim.set_state(bytes(blob))
    assert ei.value.code == -1
    sim.close()


def test_species_grows_through_pageable_uploads():
    # a species created from pageable host arrays, then given more particles than
    # its store holds: the store and the host staging area are re-allocated and
    # the upload lands whole (stored particles equal a fresh context's)
    small = W.config("c1")
    big = W.uniform_plasma((16, 16, 16), 20, 0.05, 0.05, seed=71)
    assert big.nparticles > small.nparticles
    a = PT.make_sim(small)
    a.set_particles(0, *big.species[0].arrays())
    b = PT.make_sim(big)
    assert a.count(0) == b.count(0) == big.nparticles
    pa, pb = a.get_particles(0), b.get_particles(0)
    oa, ob = np.argsort(pa["id"]), np.argsort(pb["id"])
    for k in ("id", "x", "y", "z", "ux", "uy", "uz", "w"):
        assert np.array_equal(pa[k][oa], pb[k][ob]), k
    a.step(3)
    b.step(3)
    assert PT.rel_err(a.get_fields()[0], b.get_fields()[0]) <= 1e-13
    a.close()
    b.close()


@pytest.mark.parametrize("precision,tol", [(P.FP64, 1e-15), (P.MIXED, 1e-7)])
def test_every_reader_sees_a_load_before_its_first_step(precision, tol):
    # a load bins its particles by ranks only and leaves the record moves to the next particle
    # step; reading, counting, energy, checkpoint and the tape must apply that permutation first
    import oracle as O
    wl = _two_species()
    for reader in ("particles", "count", "energy", "state", "tape"):
        sim = PT.make_sim(wl, precision=precision)
        if reader == "particles":
            for s, sp in enumerate(wl.species):
                p = sim.get_particles(s)
                o = np.argsort(p["id"])
                for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
                    assert PT.rel_err(p[k][o], getattr(sp, k)) <= tol, (reader, k)
        elif reader == "count":
            assert [sim.count(s) for s in range(2)] == [sp.n for sp in wl.species]
        elif reader == "energy":
            wk = sim.energy()[1]
            ref = O.Oracle.from_workload(wl).kinetic_energy()
            assert abs(wk - ref) <= 10 * tol * abs(ref)
        elif reader == "state":
            blob = sim.get_state()
            b = PT.make_sim(W.uniform_plasma((16, 8, 12), 1, 0.05, 0.0, seed=1), precision=precision)
            b.set_state(blob)
            sim.step(3)
            b.step(3)
            _compare(_snapshot(b, 2), _snapshot(sim, 2), 1e-12 if precision == P.FP64 else 1e-6)
            b.close()
        elif reader == "tape" and precision == P.FP64:
            wk = sim.tape_forward(2, 1)
            ora = O.Oracle.from_workload(wl)
            ora.step(2)
            assert abs(wk - ora.kinetic_energy()) <= 1e-12 * abs(wk)
        sim.close()
