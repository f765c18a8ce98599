"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2405_07898_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(md_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_binding_exports():
    names = declared_functions()
    assert names == set(binding.EXPORTS), names ^ set(binding.EXPORTS)


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = declared_functions() - exported
    assert not missing, missing
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert getattr(lib, name) is not None


def test_options_default_without_gpu():
    lib = binding.load()
    opt = binding.Options()
    lib.md_options_default(ctypes.byref(opt))
    assert opt.precision == 1 and opt.rebuild_every == 10 and opt.use_graphs == 1
    assert opt.block_size == 256 and opt.list_capacity == 0


def test_create_rejects_bad_arguments_before_touching_the_gpu():
    """Argument checks run on the host before any CUDA call."""
    from paper_2405_07898_gb300 import inputs as I
    s = I.bcc_2000_fp64()
    small = I.System(box=s.box / 3.0, pos=s.pos / 3.0, vel=s.vel, types=s.types, pot=s.pot)
    with pytest.raises(binding.MDError) as e:
        binding.MD(small, use_torch=False)
    assert e.value.status == -2  # MD_ERR_BOX
    bad = I.System(box=s.box, pos=s.pos.copy(), vel=s.vel, types=s.types, pot=s.pot)
    bad.pos[5, 1] = float("nan")
    with pytest.raises(binding.MDError) as e:
        binding.MD(bad, use_torch=False)
    assert e.value.status == -5  # MD_ERR_NONFINITE
    wrong_type = I.System(box=s.box, pos=s.pos, vel=s.vel, types=s.types + 3, pot=s.pot)
    with pytest.raises(binding.MDError) as e:
        binding.MD(wrong_type, use_torch=False)
    assert e.value.status == -1  # MD_ERR_ARG


@pytest.mark.parametrize("kw", [dict(lanes_per_atom=3), dict(block_size=100), dict(block_size=512),
                                dict(wait_limit_us=-1)])
def test_create_rejects_bad_options_before_touching_the_gpu(kw):
    from paper_2405_07898_gb300 import inputs as I
    s = I.bcc_2000_fp64()
    with pytest.raises(binding.MDError) as e:
        binding.MD(s, use_torch=False, **kw)
    assert e.value.status == -1  # MD_ERR_ARG


def test_create_rejects_out_of_range_enums():
    """persistent and precision outside their enumerations (set in the raw
    options struct, past what the Python names allow)."""
    from paper_2405_07898_gb300 import inputs as I
    s = I.bcc_2000_fp64()
    lib = binding.load()
    class Holder:
        _keep = []

    pc = binding.MD._potential_c(Holder(), s.pot)
    box = np.ascontiguousarray(s.box, dtype=np.float64)
    pos = np.ascontiguousarray(s.pos, dtype=np.float64)
    types = np.ascontiguousarray(s.types, dtype=np.int32)
    dp = ctypes.POINTER(ctypes.c_double)
    for field, value in (("persistent", 3), ("persistent", -1), ("precision", 2)):
        opt = binding.Options()
        lib.md_options_default(ctypes.byref(opt))
        setattr(opt, field, value)
        h = ctypes.c_void_p()
        rc = lib.md_create(box.ctypes.data_as(dp), s.n, pos.ctypes.data_as(dp), None,
                           types.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(pc),
                           ctypes.byref(opt), ctypes.byref(h))
        assert rc == -1, (field, rc, lib.md_last_error(None))
        assert not h.value


def test_struct_layouts_match_the_header(tmp_path):
    """Every structure the binding passes across the C ABI has the size and
    field offsets the header gives it (a small C program compiled with gcc
    prints them)."""
    pairs = [(binding.Spline, "md_spline"), (binding.PotentialC, "md_potential"),
             (binding.Options, "md_options"), (binding.Stats, "md_stats_t"),
             (binding.Profile, "md_profile_t"), (binding.Replica, "md_replica"),
             (binding.BatchInfo, "md_batch_info_t")]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "eammd.h"', "int main(void) {"]
    for cls, cname in pairs:
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cname, key, val = line.split()
            got[(cname, key)] = int(val)
    for cls, cname in pairs:
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert got[(cname, field)] == getattr(cls, field).offset, (cname, field)
