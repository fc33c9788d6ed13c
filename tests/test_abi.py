"""CPU-side checks of the boundary: the CUDA library builds for sm_103a, loads
without a GPU and exports every entry point that include/lagh.h declares; the
Python binding names them all; the seeded input generators are reproducible."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lagh.h")).read()
    return sorted(set(re.findall(r"^LH_API [^(]*?\b(lh_\w+)\(", txt, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("lh_create", "lh_force", "lh_force_sampled", "lh_mass_solve_v",
                 "lh_mass_solve_e", "lh_step", "lh_step_fixed", "lh_run_to", "lh_layout",
                 "lh_init_state"):
        assert must in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2104_11404_gb300 import build, lagh
    path = build.build()
    assert os.path.exists(path)
    L = lagh.load()
    for name in _declared():
        assert hasattr(L, name), name
    assert sorted(lagh.API_NAMES) == _declared()
    # host-only calls work without a GPU
    p = lagh.lh_default_phys()
    assert p.cfl == 0.5 and p.cfl_mu == 2.5 and p.beta1 == 0.85 and p.beta2 == 1.02
    assert p.gamma_dt == 0.8
    assert lagh.status_string(lagh.LH_ECG) == "CG did not converge"


def test_splitmix64_reference_value():
    from paper_2104_11404_gb300.workloads import SplitMix64
    # published first output of splitmix64 seeded with 0
    assert SplitMix64(0).next_u64() == 0xE220A8397B1DCDAF


def test_batch_instances_and_samples_reproducible():
    from paper_2104_11404_gb300 import workloads as W
    a = W.batch_instances(512)
    b = W.batch_instances(512)
    assert a == b and len(a) == 512
    ns = [c["n"][0] for c in a]
    assert set(ns) == set(W.BATCH_SIZES)
    assert all(0.1 <= c["blast_energy"] < 1.0 and 1.3 <= c["gamma"] < 1.67 for c in a)
    s = W.element_sample(2304, stream=7)
    assert len(s) == 116 and np.all(np.diff(s) > 0) and s[0] >= 0 and s[-1] < 2304
    assert np.array_equal(s, W.element_sample(2304, stream=7))
    assert not np.array_equal(s, W.element_sample(2304, stream=8))


def test_layout_sizes_match_oracle():
    import oracle as O
    from paper_2104_11404_gb300 import workloads as W
    for name, cfg in W.CONFIGS.items():
        nv, ne, nel = W.sizes(cfg)
        if nel > 5000:
            continue
        o = O.Oracle(dim=cfg["dim"], nx=cfg["n"][0], ny=cfg["n"][1], nz=cfg["n"][2],
                     order=cfg["order"], problem=O.UNIFORM)
        assert (o.nv, o.ne, o.nelem) == (nv, ne, nel)


STRUCTS = ["lh_mesh_desc", "lh_disc_desc", "lh_phys_desc", "lh_layout_info", "lh_run_stats",
           "lh_batch_stats", "lh_batch_tuning"]


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every ctypes mirror of a header struct has the C compiler's size and
    field offsets (a field added to one side only, or out of order, shows)."""
    import ctypes
    import shutil
    import subprocess
    from paper_2104_11404_gb300 import lagh
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lagh.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (s, s))
        for name, _ in getattr(lagh, s)._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (s, name, s, name))
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    seen = set()
    for line in out.splitlines():
        s, field, val = line.split()
        cls = getattr(lagh, s)
        if field == "sizeof":
            assert ctypes.sizeof(cls) == int(val), s
        else:
            assert getattr(cls, field).offset == int(val), (s, field)
        seen.add(s)
    assert seen == set(STRUCTS)


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the shared library missing, loading raises."""
    from paper_2104_11404_gb300 import lagh
    monkeypatch.setattr(lagh, "_lib", None)
    monkeypatch.setattr(lagh, "LIB_PATH", str(tmp_path / "missing" / "liblagh.so"))
    with pytest.raises(RuntimeError):
        lagh.load()


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_compiles_strictly_as_c_and_cpp(tmp_path, lang, std):
    """The boundary header is plain C: it compiles as C99 and as C++ with
    every warning an error, for callers outside this package."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no compiler")
    src = tmp_path / ("use.c" if lang == "c" else "use.cpp")
    src.write_text('#include "lagh.h"\n'
                   "int main(void) { lh_phys_desc p; lh_default_phys(&p); return p.cg_maxit < 0; }\n")
    subprocess.run([cc, std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                    os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "use.o")],
                   check=True)


def test_library_c_exports_are_exactly_the_header_entry_points():
    """Every exported C-linkage symbol of the library is an lh_* entry point of
    include/lagh.h, and every one of those is exported (names from nm)."""
    import shutil
    import subprocess
    from paper_2104_11404_gb300 import build
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("no nm")
    path = build.build()
    out = subprocess.run([nm, "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    names = [f[-1] for f in (l.split() for l in out.splitlines()) if len(f) >= 3]
    c_names = sorted(n for n in names if not n.startswith("_Z"))
    assert c_names == _declared()


def test_wrappers_reject_unknown_precision_overrides_and_tuning_keys():
    """Misspelt options fail at once, before any device call (a ctypes struct
    would otherwise take an unknown name as a plain Python attribute)."""
    from paper_2104_11404_gb300 import lagh
    from paper_2104_11404_gb300 import workloads as W
    from paper_2104_11404_gb300.batch import Batch
    from paper_2104_11404_gb300.hydro import Hydro, descriptors, precision_id
    cfg = W.CONFIGS["sedov2d_8"]
    assert precision_id("fp64") == lagh.LH_FP64 and precision_id("mixed") == lagh.LH_MIXED
    with pytest.raises(ValueError):
        precision_id("fp32")
    with pytest.raises(ValueError):
        Hydro(cfg, precision="fp32")
    _, _, phys = descriptors(cfg, phys_overrides={"cg_tiles": -1, "cg_cluster": 1})
    assert phys.cg_tiles == -1 and phys.cg_cluster == 1
    with pytest.raises(KeyError):
        descriptors(cfg, phys_overrides={"cg_tile": -1})
    with pytest.raises(KeyError):
        Batch([cfg], tuning={"thread": 256})
    with pytest.raises(ValueError):
        Batch([cfg], precision="single")


def test_lane_probe_rejects_lane_counts_outside_a_warp():
    """lh_peak_probe_lanes checks its arguments before any CUDA call."""
    import ctypes
    from paper_2104_11404_gb300 import lagh
    L = lagh.load()
    sink = (ctypes.c_double * 8)()
    for lanes in (0, 33, -1):
        st = L.lh_peak_probe_lanes(1, lanes, 10, ctypes.cast(sink, ctypes.c_void_p), None, None)
        assert st == lagh.LH_EINVAL
