"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/metad.h declares.  No compute call is made: these run without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def metad():
    from paper_2510_06873_gb300 import build
    build.build()
    from paper_2510_06873_gb300 import metad as m
    m.lib()
    return m


def declared_functions():
    names = set()
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(metad_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(metad):
    names = declared_functions()
    assert len(names) >= 20
    lib = metad.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    unbound = [n for n in names if n not in metad._SIGS]
    assert not unbound, unbound


def test_params_struct_round_trips(metad):
    p = metad.metad_params_default()
    assert ctypes.sizeof(metad.metad_params) == 240
    assert (p.n_atoms, p.n_cv, p.sw_n, p.sw_m, p.stretch, p.cn_pairs) == (1, 2, 6, 12, 1, 1)
    assert (p.rc, p.r0, p.w0, p.biasfactor, p.temperature) == (3.5, 2.5, 1.0, 10.0, 300.0)
    assert list(p.sigma) == [0.05, 0.02] and p.kB == 0.0083144626
    assert p.hill_capacity == 65536 and p.max_neighbors == 64 and list(p.grid_n) == [200, 200]
    assert p.skin == 1.0
    assert p.cv_kind == metad.METAD_CV_COORDINATION and p.softmin_beta == 0.0
    assert (p.lattice_cvs, p.virial) == (0, 0) and list(p.sigma_lattice) == [0.1, 0.1, 0.1]


@pytest.mark.parametrize("field,value", [("n_atoms", 0), ("n_cv", 3), ("box", 6.9), ("sigma", 0.0),
                                         ("biasfactor", 1.0), ("precision", 2), ("sw_m", 6),
                                         ("hill_capacity", 0), ("max_neighbors", -1),
                                         ("skin", -0.5)])
def test_invalid_params_rejected_before_any_device_call(metad, field, value):
    p = metad.metad_params_default()
    p.n_atoms = 100
    if field == "box":
        p.box[0] = value
    elif field == "sigma":
        p.sigma[0] = value
    else:
        setattr(p, field, value)
    with pytest.raises(metad.MetadError) as e:
        metad.metad_create(p)
    assert e.value.status == metad.METAD_ERR_INVALID


def test_grid_needs_two_cvs(metad):
    p = metad.params_for(10, [10, 10, 10], n_cv=1, sigma=(0.05,), grid=((200, 200), (0, 0), (1, 1)))
    with pytest.raises(metad.MetadError) as e:
        metad.metad_create(p)
    assert e.value.status == metad.METAD_ERR_INVALID


def test_status_strings_and_stage_names(metad):
    assert metad.status_string(0) == "ok"
    assert metad.status_string(4) == "capacity exceeded"
    assert [metad.metad_stage_name(k) for k in range(metad.METAD_NUM_STAGES)][7:9] == ["force_pairs", "force_gather"]
    assert metad.lib().metad_destroy(None) == 0


def test_package_import_does_not_load_oracle():
    import subprocess
    import sys
    code = ("import sys; import paper_2510_06873_gb300.metad as m; m.lib(); "
            "assert 'oracle' not in sys.modules, 'oracle imported by the library path'")
    subprocess.check_call([sys.executable, "-c", code], cwd=ROOT)


def test_estimate_bytes_needs_no_gpu_and_grows_with_size(metad):
    small = metad.metad_estimate_bytes(metad.params_for(1000, [23.2, 23.2, 23.2]))
    big = metad.metad_estimate_bytes(metad.params_for(100_000, [106.0, 106.0, 106.0]))
    assert 0 < small < big
    # a few KB per atom (neighbour rows, pair slots and cross terms, Verlet
    # rows, records)
    per_atom = (big - small) / 99_000
    assert 1000 < per_atom < 4500, per_atom
    with pytest.raises(metad.MetadError) as e:
        metad.metad_estimate_bytes(metad.params_for(10, [1.0, 10.0, 10.0]))
    assert e.value.status == metad.METAD_ERR_INVALID


def test_row_capacity_is_a_multiple_of_four(metad):
    """Rows hold a multiple of four (j, w) entries (0 asks for 64), so an even
    entry always begins a 16 B pair inside its row: the Q6 and adjoint passes
    read row entries two per load.  The creation path and the estimate share
    the rounding; the estimate shows it without a GPU."""
    def est(m):
        p = metad.params_for(20_000, [62.0, 62.0, 62.0])
        p.max_neighbors = m
        return metad.metad_estimate_bytes(p)

    assert est(5) == est(6) == est(7) == est(8) < est(9) == est(12)
    assert est(0) == est(64) == est(61)


def test_batch_entry_points_reject_null_without_a_gpu(metad):
    import ctypes
    L = metad.lib()
    out = ctypes.c_void_p()
    assert L.metad_batch_create(None, 1, ctypes.byref(out)) == metad.METAD_ERR_INVALID
    arr = (ctypes.c_void_p * 1)(None)
    assert L.metad_batch_create(arr, 1, ctypes.byref(out)) == metad.METAD_ERR_INVALID
    assert L.metad_batch_create(arr, 0, ctypes.byref(out)) == metad.METAD_ERR_INVALID
    assert L.metad_batch_step(None, None, None, 0, None, None) == metad.METAD_ERR_INVALID
    assert L.metad_batch_read(None, None, None) == metad.METAD_ERR_INVALID
    assert L.metad_batch_set_tile(None, 0) == metad.METAD_ERR_INVALID
    assert L.metad_batch_destroy(None) == metad.METAD_OK


@pytest.mark.parametrize("kind,field,value", [("torsion", "n_atoms", 3), ("torsion", "grid_on", 1),
                                              ("nearest", "softmin_beta", -1.0), ("nearest", "box", 0.0),
                                              ("coordination", "cv_kind", 3)])
def test_small_cv_families_reject_bad_params(metad, kind, field, value):
    p = metad.params_for(22, [24.0, 24.0, 24.0], sigma=(0.35, 0.35), cv_kind=kind)
    if field == "box":
        p.box[1] = value
    elif field == "grid_on":
        p.grid_on, p.grid_n[0], p.grid_n[1], p.grid_hi[0], p.grid_hi[1] = 1, 10, 10, 1.0, 1.0
    else:
        setattr(p, field, value)
    with pytest.raises(metad.MetadError) as e:
        metad.metad_estimate_bytes(p)
    assert e.value.status == metad.METAD_ERR_INVALID


def test_small_cv_families_allocate_no_neighbour_state(metad):
    # a box far below 2 rc is fine without a neighbour list
    p = metad.params_for(22, [5.0, 5.0, 5.0], sigma=(0.35, 0.35), cv_kind="torsion", hill_capacity=1000)
    b = metad.metad_estimate_bytes(p)
    # hills (centres twice: live + staging), hill-block partials, scalars; no per-atom rows
    assert b < 128 * 1024, b
    big = metad.params_for(100_000, [50.0, 50.0, 50.0], sigma=(0.1,), n_cv=1, cv_kind="nearest",
                           hill_capacity=1000)
    assert metad.metad_estimate_bytes(big) < 100_000 * 16 + 64 * 1024


@pytest.mark.parametrize("field,value", [("lattice_cvs", 2), ("virial", -1), ("sigma_lattice", 0.0),
                                         ("grid_on", 1), ("cv_kind", 1)])
def test_lattice_cvs_reject_bad_params(metad, field, value):
    p = metad.params_for(5000, [40.0, 40.0, 40.0], lattice_cvs=True)
    if field == "sigma_lattice":
        p.sigma_lattice[2] = value
    elif field == "grid_on":
        p.grid_on, p.grid_n[0], p.grid_n[1], p.grid_hi[0], p.grid_hi[1] = 1, 10, 10, 1.0, 1.0
    else:
        setattr(p, field, value)
    with pytest.raises(metad.MetadError) as e:
        metad.metad_estimate_bytes(p)
    assert e.value.status == metad.METAD_ERR_INVALID


def test_lattice_hills_take_five_doubles(metad):
    base = metad.metad_estimate_bytes(metad.params_for(5000, [40.0, 40.0, 40.0], hill_capacity=10000))
    lat = metad.metad_estimate_bytes(metad.params_for(5000, [40.0, 40.0, 40.0], hill_capacity=10000,
                                                      lattice_cvs=True))
    # centres (live + staging) grow from 2 to 5 doubles per hill
    assert lat - base == 2 * 3 * 8 * 10001
