"""GPU tests of lbib_save / lbib_load (checkpoint and resume of a context's
full step state): resuming from a saved state reproduces the uninterrupted run
bit for bit (populations, markers, bonds) in every precision; a state saved by
another set-up, a truncated file and a non-state file are refused with the
context untouched."""
import os

import numpy as np
import pytest

from paper_1907_00080_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_00080_gb300 import build, lbib
    build.build()
    lbib.load()


def lb():
    from paper_1907_00080_gb300 import lbib
    return lbib


@pytest.mark.parametrize("case,prec", [("capillary", "f64"), ("capillary", "f32"), ("capillary", "f16"),
                                       ("capsule", "f64"), ("capsule", "f32")])
def test_resume_reproduces_the_run(case, prec, tmp_path):
    """100 steps, save, 60 more; a fresh context loads the file and steps 60:
    the coarse capillary, and the capsule with the stress bond kinetics (bonds
    form and break across the save)."""
    L = lb()
    if case == "capillary":
        wl = inputs.capillary(precision=prec, seed=3)
    else:
        wl = inputs.capsule_128x32(prec, bonds="stress")
    path = str(tmp_path / "state.lbib")
    a = L.Simulation(wl)
    a.step(100)
    a.save(path)
    b100 = a.bonds()
    a.step(60)
    ref = (a.populations(), a.markers(), a.bonds())
    a.close()
    b = L.Simulation(wl)
    b.load_state(path)
    assert L.lbib_step_count(b.ctx) == 100
    b.step(60)
    got = (b.populations(), b.markers(), b.bonds())
    b.close()
    for x, y in zip(got, ref):
        np.testing.assert_array_equal(x, y)
    if case == "capsule":
        assert (b100 >= 0).any() or (ref[2] >= 0).any()


def test_load_into_the_same_context_rewinds_it(tmp_path):
    L = lb()
    wl = inputs.capsule_128x32("f64", bonds="stress")
    path = str(tmp_path / "s.lbib")
    s = L.Simulation(wl)
    s.step(40)
    s.save(path)
    x40 = s.markers()
    s.step(25)
    x65 = s.markers()
    s.load_state(path)
    np.testing.assert_array_equal(s.markers(), x40)
    s.step(25)
    np.testing.assert_array_equal(s.markers(), x65)
    s.close()


def test_other_set_ups_and_bad_files_are_refused(tmp_path):
    L = lb()
    path = str(tmp_path / "s.lbib")
    s = L.Simulation(inputs.capsule_128x32("f64"))
    s.step(5)
    s.save(path)
    x = s.markers()
    # other precision, other lattice, other body force
    for wl in (inputs.capsule_128x32("f32"), inputs.capillary(nx=128, ny=32, n_rbc=0, n_carriers=1, precision="f64")):
        o = L.Simulation(wl)
        with pytest.raises(L.LbibError) as ei:
            o.load_state(path)
        assert ei.value.status == L.LBIB_E_INVALID
        o.close()
    # truncated file and a file that is not a state: refused, context unchanged
    with open(path, "rb") as fh:
        blob = fh.read()
    short = str(tmp_path / "short.lbib")
    with open(short, "wb") as fh:
        fh.write(blob[: len(blob) // 2])
    junk = str(tmp_path / "junk.lbib")
    with open(junk, "wb") as fh:
        fh.write(os.urandom(256))
    for bad in (short, junk, str(tmp_path / "missing.lbib")):
        with pytest.raises(L.LbibError) as ei:
            s.load_state(bad)
        assert ei.value.status == L.LBIB_E_INVALID
    np.testing.assert_array_equal(s.markers(), x)
    with pytest.raises(L.LbibError) as ei:
        s.save(str(tmp_path / "no_such_dir" / "s.lbib"))
    assert ei.value.status == L.LBIB_E_INVALID
    s.close()


def test_same_sizes_other_parameters_are_refused(tmp_path):
    """A state only loads into the set-up that saved it: the same lattice and
    the same numbers of membranes, vertices, ligands and receptors, but another
    k_s, k_b, ligand element, receptor position, sigma, density or membrane
    kind is refused, and so is a file with bytes after its last part."""
    import dataclasses
    L = lb()
    path = str(tmp_path / "s.lbib")
    base = inputs.capsule_128x32("f64", bonds="stress")
    s = L.Simulation(base)
    s.step(5)
    s.save(path)

    def variant(**kw):
        wl = dataclasses.replace(base)
        mem = dataclasses.replace(base.membranes[0], **{k: v for k, v in kw.items() if k in ("ks", "kb", "kind", "ligands", "rho_p")})
        wl.membranes = [mem]
        if "receptors" in kw:
            wl.receptors = kw["receptors"]
        if "sigma_lu" in kw:
            wl.sigma_lu = kw["sigma_lu"]
        return wl

    rec = base.receptors.copy()
    rec[3, 0] += 0.25
    lig = base.membranes[0].ligands.copy()
    lig[-1] = 0
    lig[0] = 31
    for wl in (variant(ks=0.051), variant(kb=0.004), variant(receptors=rec), variant(ligands=lig),
               variant(sigma_lu=2 * base.sigma_lu), variant(kind=1)):
        o = L.Simulation(wl)
        with pytest.raises(L.LbibError) as ei:
            o.load_state(path)
        assert ei.value.status == L.LBIB_E_INVALID
        o.close()
    # the set-up that saved it loads it
    o = L.Simulation(base)
    o.load_state(path)
    np.testing.assert_array_equal(o.markers(), s.markers())
    o.close()
    # a trailing byte is refused
    longer = str(tmp_path / "long.lbib")
    with open(path, "rb") as fh, open(longer, "wb") as out:
        out.write(fh.read() + b"\0")
    with pytest.raises(L.LbibError) as ei:
        s.load_state(longer)
    assert ei.value.status == L.LBIB_E_INVALID
    s.close()
