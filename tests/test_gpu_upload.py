"""Double-buffered particle uploads (pic_upload_particles, pic_set_particles_uploaded).

* An upload copied while the context keeps stepping its current particles,
  then installed, gives the same store and the same next steps as a
  synchronous pic_set_particles at that point (the current particles are not
  touched by the upload).
* The pipelined loop (install step i's upload, start step i+1's, step, read
  the energy) follows the synchronous loop step for step.
* An upload larger than the species' store grows both; an upload replaced
  before installation is dropped; installing with nothing pending, or
  uploading to an immobile species, is refused and leaves the context usable.
* Device arrays upload like page-locked host arrays.
"""
import numpy as np
import pytest

from paper_1608_01009_gb300 import pic as P
from paper_1608_01009_gb300 import workloads as W
from tests import parity as PT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pinned(arrays):
    out = []
    for a in arrays:
        t = torch.empty(a.shape[0], dtype=torch.float64, pin_memory=True)
        t.numpy()[:] = a
        out.append(t.numpy())
    return out


def _same_particles(a, b, tol=0.0):
    """Equal stores: bit for bit right after a load (tol = 0); after steps the
    fields, and so the particles, differ by the order of the floating-point
    atomics (tol)."""
    pa, pb = a.get_particles(0), b.get_particles(0)
    oa, ob = np.argsort(pa["id"]), np.argsort(pb["id"])
    assert np.array_equal(pa["id"][oa], pb["id"][ob])
    for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
        if tol == 0.0:
            assert np.array_equal(pa[k][oa], pb[k][ob]), k
        else:
            assert PT.rel_err(pb[k][ob], pa[k][oa]) <= tol, k


@pytest.mark.parametrize("precision,tol", [(P.FP64, 1e-12), (P.MIXED, 1e-5)])
def test_upload_while_stepping_then_install(precision, tol):
    # same operations on both sides; they differ only in the order of the
    # floating-point atomics (FP32 shared-memory sums in the mixed path)
    wl = W.config("c1")
    new = W.uniform_plasma((16, 16, 16), 12, 0.05, 0.08, seed=83)  # more particles than the store holds
    arrs = _pinned(new.species[0].arrays())
    a = PT.make_sim(wl, precision=precision)
    b = PT.make_sim(wl, precision=precision)
    b.upload_particles(0, *arrs)
    a.step(2)
    b.step(2)  # the current particles step while the upload is copied
    a.set_particles(0, *arrs)
    b.set_particles_uploaded(0)
    _same_particles(a, b)
    a.step(3)
    b.step(3)
    b.sync()
    assert PT.rel_err(b.get_fields()[0], a.get_fields()[0]) <= tol
    assert abs(b.energy()[1] - a.energy()[1]) <= tol * a.energy()[1]
    a.close()
    b.close()


def test_pipelined_loop_follows_the_synchronous_loop():
    wl = W.config("c1")
    arrs = _pinned(wl.species[0].arrays())
    a = PT.make_sim(wl)
    b = PT.make_sim(wl)
    b.upload_particles(0, *arrs)
    for i in range(4):
        a.set_particles(0, *arrs)
        a.step(1)
        b.set_particles_uploaded(0)
        if i < 3:
            b.upload_particles(0, *arrs)  # the next step's set, copied while this step runs
        b.step(1)
        ea, eb = a.energy(), b.energy()
        assert abs(eb[0] - ea[0]) <= 1e-12 * abs(ea[0]) + 1e-300 and abs(eb[1] - ea[1]) <= 1e-12 * ea[1]
    _same_particles(a, b, tol=1e-12)
    a.close()
    b.close()


def test_replaced_upload_and_refusals():
    wl = W.config("c1")
    other = W.uniform_plasma((16, 16, 16), 3, 0.05, 0.05, seed=84)
    sim = PT.make_sim(wl)
    with pytest.raises(P.PicError) as ei:
        sim.set_particles_uploaded(0)
    assert ei.value.code == -7  # PIC_ERR_STATE: nothing pending
    sim.upload_particles(0, *_pinned(other.species[0].arrays()))
    sim.upload_particles(0, *_pinned(wl.species[0].arrays()))  # replaces the first
    sim.set_particles_uploaded(0)
    assert sim.count(0) == wl.nparticles
    with pytest.raises(P.PicError) as ei:
        sim.set_particles_uploaded(0)  # consumed
    assert ei.value.code == -7
    ion = sim.add_species(1.0, 1836.0, *wl.species[0].arrays(), immobile=True)
    with pytest.raises(P.PicError) as ei:
        sim.upload_particles(ion, *wl.species[0].arrays())
    assert ei.value.code == -1  # PIC_ERR_ARG
    ref = PT.make_sim(wl)
    _same_particles(sim, ref)
    sim.step(2)
    ref.step(2)
    assert PT.rel_err(sim.get_fields()[0], ref.get_fields()[0]) <= 1e-12
    sim.close()
    ref.close()


def test_upload_from_device_tensors():
    # device arrays (torch tensors on the GPU) go through the same upload area
    wl = W.config("c1")
    new = W.uniform_plasma((16, 16, 16), 10, 0.05, 0.06, seed=85)
    arrs = new.species[0].arrays()
    a = PT.make_sim(wl)
    b = PT.make_sim(wl)
    a.upload_particles(0, *_pinned(arrs))
    b.upload_particles(0, *[torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in arrs])
    a.set_particles_uploaded(0)
    b.set_particles_uploaded(0)
    _same_particles(a, b)
    a.close()
    b.close()
