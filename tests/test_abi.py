"""CPU-side checks of the C ABI: the library loads without a GPU, exports
every function declared in include/hff.h, and validates configurations and
plans memory on the host (no device calls)."""
import os
import re

import pytest

from paper_2406_14512_gb300 import build as hff_build
from paper_2406_14512_gb300 import hff, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    hff_build.build()
    return hff.load()


def declared():
    src = open(os.path.join(ROOT, "include", "hff.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(hff_[a-z_]+)\s*\(", src, re.M)))


def test_header_declares_the_binding_symbols():
    assert declared() == sorted(hff.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_plan_sizes_scale_with_grid_and_capacity(lib):
    c1 = hff.config_struct(dict(workloads.config("c1"), capacity=300_000))
    b1 = hff.hff_plan(c1)
    c2 = hff.config_struct(dict(workloads.config("c1"), capacity=600_000))
    b2 = hff.hff_plan(c2)
    assert b2 > b1 > 0
    c3 = workloads.config("c3")
    c3["capacity"] = int(1.1 * c3["n_pairs"])
    b3 = hff.hff_plan(hff.config_struct(c3))
    # 2 species x 1.65e8 slots x 28 B x 2 sort buffers, 16 B of sort keys per
    # slot, and about 1.5 GB of fields: ~23 GB of the 280 GB of HBM
    assert 15e9 < b3 < 40e9, b3


def test_stellar_row_return_takes_the_separate_field_passes(lib):
    """ff_delta_only = 2 exists in the separate field kernels only: on a grid
    where the automatic choice is the fused pass (4096^2), the plan then
    reserves no halo snapshot for it, and the fused pass's own explicit
    request plans the snapshot."""
    c = dict(workloads.config("c3"), capacity=1000, tile_r=16, tile_t=24, sort_every=12)
    fused = hff.hff_plan(hff.config_struct(c))
    split = hff.hff_plan(hff.config_struct(dict(c, field_pass=2)))
    auto2 = hff.hff_plan(hff.config_struct(dict(c, ff_delta_only=2)))
    assert fused > split and auto2 == split, (fused, split, auto2)


@pytest.mark.parametrize("bad", [dict(nr=4), dict(courant=1.5), dict(sort_every=33), dict(n_breaks_bad=True),
                                 dict(r_abs="one_cell_inside"), dict(precision_bad=True),
                                 dict(field_pass_bad=True), dict(ff_delta_only=3),
                                 dict(ff_delta_only=2, field_pass=1)])
def test_invalid_configs_are_rejected(lib, bad):
    cfg = workloads.config("small_pic")
    cfg.update(capacity=10)
    c = hff.config_struct(cfg)
    if "nr" in bad:
        c.nr = bad["nr"]
    if "courant" in bad:
        c.courant = bad["courant"]
    if "sort_every" in bad:
        c.sort_every = bad["sort_every"]
    if "n_breaks_bad" in bad:
        c.n_breaks = 2
        c.psi_break[0], c.psi_break[1] = 2.0, 1.0
    if "r_abs" in bad:  # inside r_max but closer than 3 cells to it (r_abs >= r_max means no absorber)
        c.r_abs = c.r_max * (c.r_max / c.r_min) ** (-1.0 / c.nr)
    if "precision_bad" in bad:
        c.precision = 7
    if "field_pass_bad" in bad:
        c.field_pass = 3
    if "ff_delta_only" in bad:  # 2 (the stellar-row return) exists in the separate passes only
        c.ff_delta_only = bad["ff_delta_only"]
        c.field_pass = bad.get("field_pass", 0)
    with pytest.raises(hff.HffError) as e:
        hff.hff_plan(c)
    assert e.value.code == hff.HFF_ERR_ARG
    assert hff.hff_last_error()


def test_header_is_plain_c_and_cxx(tmp_path):
    """include/hff.h compiles as C99 and as C++17 on its own, and a C caller
    can name every declared function (link-free: declarations only)."""
    import shutil
    import subprocess
    if not shutil.which("gcc") or not shutil.which("g++"):
        pytest.skip("no host C compiler")
    hdr = os.path.join(ROOT, "include", "hff.h")
    for cc, lang, std in (("gcc", "c", "-std=c99"), ("g++", "c++", "-std=c++17")):
        subprocess.run([cc, "-fsyntax-only", "-Wall", "-Wextra", "-Werror", "-x", lang, std, hdr], check=True)
    src = tmp_path / "use.c"
    src.write_text('#include "hff.h"\n'
                   "int main(void) {\n"
                   "  hff_config c = {0};\n  size_t b = 0;\n"
                   "  void *f[] = {(void *)hff_plan, (void *)hff_init, (void *)hff_step, (void *)hff_fields,\n"
                   "               (void *)hff_particles, (void *)hff_diagnostics, (void *)hff_checkpoint_save,\n"
                   "               (void *)hff_spectrum, (void *)hff_tile_order_noalloc};\n"
                   "  (void)f;\n  return hff_plan(&c, 1, &b) == 0 ? 1 : 0;\n}\n")
    subprocess.run(["gcc", "-fsyntax-only", "-Wall", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src)],
                   check=True)


def test_binding_struct_layouts_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and the field
    offsets of its C declaration (a C program prints them)."""
    import ctypes
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no host C compiler")
    structs = [hff.hff_config, hff.hff_info, hff.hff_particle_view, hff.hff_diag]
    body = []
    for st in structs:
        name = st.__name__
        body.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f in st._fields_:
            body.append(f'  printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "hff.h"\nint main(void) {\n'
                   + "\n".join(body) + "\n  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in structs:
        assert got[(st.__name__, "size")] == ctypes.sizeof(st), st.__name__
        for f in st._fields_:
            assert got[(st.__name__, f[0])] == getattr(st, f[0]).offset, (st.__name__, f[0])


def test_info_ring_depth_matches_the_header():
    import re
    text = open(os.path.join(ROOT, "include", "hff.h")).read()
    m = re.search(r"#define\s+HFF_INFO_RING\s+(\d+)", text)
    assert m and int(m.group(1)) == hff.INFO_RING
