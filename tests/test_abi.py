"""The C ABI library builds, loads, exports every symbol the header declares, and its host-side
validation works without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kbc_lb.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(lb_[a-z_]+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1507_02518_gb300 import build, lb
    build.build()
    return lb.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lb_create", "lb_init_field", "lb_step", "lb_moments", "lb_diagnostics",
                 "lb_get_populations", "lb_set_populations", "lb_batch_step"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1507_02518_gb300 import lb
    names = declared_functions()
    for n in names:
        assert hasattr(lib, n), "libkbc.so does not export %s" % n
    assert sorted(lb.SYMBOLS) == names


def test_required_bytes_and_validation(lib):
    from paper_1507_02518_gb300 import lb
    c = lb.make_config(32, storage="f64", scheme="pull")
    need_pull = lb.lb_required_bytes(c)
    assert need_pull >= 2 * 27 * 32 ** 3 * 8
    c_aa = lb.make_config(32, storage="f64", scheme="aa")
    assert lb.lb_required_bytes(c_aa) < need_pull
    assert lb.lb_required_bytes(lb.make_config(32, storage="f16")) < lb.lb_required_bytes(
        lb.make_config(32, storage="f32"))
    for bad in (lb.make_config(2), lb.make_config(32, nu=0.0), lb.make_config(32, nu=-1.0),
                lb.make_config(1 << 11, 1 << 10, 1 << 10)):
        assert lb.lb_required_bytes(bad) == 0
    c_bad = lb.make_config(32)
    c_bad.variant = 8
    assert lb.lb_required_bytes(c_bad) == 0


def test_slab_and_mask_sizes_on_host(lib):
    """A slab context holds its planes plus one halo plane per side, the FP64 re-collision mask
    (one bit per node), and four face buffers of 9 nx ny stored values; invalid slabs size to 0."""
    from paper_1507_02518_gb300 import lb
    nx, ny, nz = 24, 16, 12
    g = lb.make_config(nx, ny, nz, storage="f32", scheme="aa")
    for k in (1, 3, nz):
        need = lb.lb_slab_required_bytes(g, k)
        box = lb.lb_required_bytes(lb.make_config(nx, ny, k + 2, storage="f32", scheme="aa"))
        assert need >= box + 4 * 9 * nx * ny * 4
        assert need >= 27 * nx * ny * (k + 2) * 4 + (nx * ny * (k + 2) + 31) // 32 * 4
    for bad in (0, -1, nz + 1):
        assert lb.lb_slab_required_bytes(g, bad) == 0
    # the mask grows with the node count: one bit per node on top of the populations
    small = lb.lb_required_bytes(lb.make_config(32, storage="f16", scheme="aa"))
    assert small >= 27 * 32 ** 3 * 2 + 32 ** 3 // 8 + 32 ** 3 * 4


def test_create_rejects_bad_arguments_on_host(lib):
    from paper_1507_02518_gb300 import lb
    with pytest.raises(lb.LBError) as e:
        lb.lb_create(lb.make_config(2), 256, 1 << 30, 0)
    assert e.value.status == lb.LB_ERR_INVALID_ARG
    with pytest.raises(lb.LBError) as e:
        lb.lb_create(lb.make_config(32), 256, 100, 0)
    assert e.value.status == lb.LB_ERR_OOM
    with pytest.raises(lb.LBError) as e:
        lb.lb_create(lb.make_config(32), 0, 1 << 30, 0)
    assert e.value.status == lb.LB_ERR_INVALID_ARG
    with pytest.raises(lb.LBError) as e:
        lb.lb_create(lb.make_config(32), 100, 1 << 30, 0)   # misaligned
    assert e.value.status == lb.LB_ERR_INVALID_ARG
    with pytest.raises(lb.LBError) as e:
        lb.lb_batch_create([], 256, 1 << 30, 0)
    assert e.value.status == lb.LB_ERR_INVALID_ARG


def test_null_handles_are_rejected(lib):
    assert lib.lb_step(None, 1) == 1
    assert lib.lb_destroy(None) == 1
    assert lib.lb_batch_step(None, 1) == 1
    assert lib.lb_time(None) == -1


def test_equilibrium_choice_is_validated(lib):
    from paper_1507_02518_gb300 import lb
    assert lb.lb_required_bytes(lb.make_config(32, equilibrium="poly2")) > 0
    c = lb.make_config(32)
    c.equilibrium = 2
    assert lb.lb_required_bytes(c) == 0
    with pytest.raises(lb.LBError) as e:     # refused on the host, before any device call
        lb.lb_create(lb.make_config(32, gamma="exact", equilibrium="poly2"), 256, 1 << 30, 0)
    assert e.value.status == lb.LB_ERR_UNSUPPORTED


def test_binding_structs_and_enums_match_the_header(tmp_path):
    """The ctypes mirrors of lb_config, lb_diag and lb_gap have the C layout (size and every
    field offset, as gcc lays out the header), and the binding's enum values are the header's."""
    import subprocess
    from paper_1507_02518_gb300 import lb
    structs = {"lb_config": lb.lb_config, "lb_diag": lb.lb_diag, "lb_gap": lb.lb_gap}
    enums = ["LB_OK", "LB_ERR_INVALID_ARG", "LB_ERR_OOM", "LB_ERR_CUDA", "LB_ERR_NONFINITE",
             "LB_ERR_TIMEOUT", "LB_ERR_UNSUPPORTED", "LB_S_D", "LB_S_DT", "LB_S_DQ", "LB_S_DTQ",
             "LB_S_CD", "LB_S_CDT", "LB_S_CDQ", "LB_S_CDTQ", "LB_GAMMA_ESTIMATE", "LB_GAMMA_LBGK",
             "LB_GAMMA_RLB", "LB_GAMMA_EXACT", "LB_F64", "LB_F32", "LB_F16", "LB_PULL", "LB_AA",
             "LB_EQ_PRODUCT", "LB_EQ_POLY2", "LB_KERNEL_AUTO", "LB_KERNEL_DIRECT",
             "LB_KERNEL_STAGED", "LB_KERNEL_PERSISTENT", "LB_KERNEL_PACKED", "LB_KERNEL_ROWS", "LB_KERNEL_ADJ"]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "kbc_lb.h"',
             "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));'
                         % (name, field, name, field))
    for e in enums:
        lines.append('printf("enum %s %%d\\n", (int)%s);' % (e, e))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        *key, value = line.split()
        got[tuple(key)] = int(value)
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
    for e in enums:
        assert got[("enum", e)] == getattr(lb, e), e
