"""The C-ABI library loads and exports every entry point declared in include/mgh.h (CPU only:
no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mgh.h")
LIB = os.path.join(ROOT, "paper_2107_03679_gb300", "libmgh.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mgh_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__ as g
        g.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mgh_create", "mgh_destroy", "mgh_set_contrast", "mgh_rhs", "mgh_apply",
                     "mgh_precondition", "mgh_solve", "mgh_forward", "mgh_gradient", "mgh_crop",
                     "mgh_sample", "mgh_misfit", "mgh_workspace_bytes", "mgh_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    import paper_2107_03679_gb300.capi as capi
    assert sorted(capi.EXPORTED) == declared_functions()
    for n in declared_functions():
        assert callable(getattr(capi, n))


def test_host_only_entry_points(lib):
    """Parameter validation and sizing run on the host without touching a GPU."""
    import paper_2107_03679_gb300.capi as capi
    p = capi.mgh_default_params()
    assert p.nx_int == 128 and p.levels == 4 and p.restart == 20
    assert capi.mgh_workspace_bytes(p) > 16 * (p.nx_int + 2 * p.abl) ** 2 * (p.restart + 1)
    bad = capi.mgh_default_params()
    bad.levels = 1
    with pytest.raises(capi.MGHError):
        capi.mgh_workspace_bytes(bad)
    ok = capi.mgh_default_params()
    ok.levels = 2           # coarsest 80x80 = 6400 unknowns: within the 8192 of the dense inverse
    assert capi.mgh_workspace_bytes(ok) > 16 * 6400 * 6400
    bad = capi.mgh_default_params()
    bad.nx_int = bad.ny_int = 200
    bad.levels = 2          # coarsest 116x116 = 13456 unknowns > dense-inverse limit
    with pytest.raises(capi.MGHError):
        capi.mgh_workspace_bytes(bad)
    assert capi.mgh_status_string(capi.MGH_NOT_CONVERGED) == "not converged"
    # the s-step engine holds its Gram sums in registers: restart 1..8 on the mixed path
    ss = capi.mgh_default_params()
    ss.precision, ss.arnoldi, ss.restart = capi.MGH_PREC_MIXED32, capi.MGH_ARNOLDI_SSTEP, 8
    assert capi.mgh_workspace_bytes(ss) > 0
    ss.restart = 9
    with pytest.raises(capi.MGHError):
        capi.mgh_workspace_bytes(ss)
    ss.arnoldi = 3
    with pytest.raises(capi.MGHError):
        capi.mgh_workspace_bytes(ss)
    # Bi-CGSTAB keeps its six FP64 vectors in the GMRES workspace: restart >= 5
    bc = capi.mgh_default_params()
    bc.krylov = capi.MGH_KRYLOV_BICGSTAB
    assert capi.mgh_workspace_bytes(bc) > 0
    bc.restart = 4
    with pytest.raises(capi.MGHError):
        capi.mgh_workspace_bytes(bc)
    bc.restart, bc.krylov = 8, 2
    with pytest.raises(capi.MGHError):
        capi.mgh_workspace_bytes(bc)
    # FP16 storage (MGH_PREC_MIXED16): s-step FGMRES, even width, a sweep on each side of level 0
    hs = capi.mgh_default_params()
    hs.precision, hs.arnoldi, hs.restart = capi.MGH_PREC_MIXED16, capi.MGH_ARNOLDI_SSTEP, 8
    assert capi.mgh_workspace_bytes(hs) > 0
    for field, value in (("arnoldi", capi.MGH_ARNOLDI_DF), ("krylov", capi.MGH_KRYLOV_BICGSTAB), ("nx_int", 129),
                         ("nu2", 0)):
        bad = capi.mgh_default_params()
        bad.precision, bad.arnoldi, bad.restart = capi.MGH_PREC_MIXED16, capi.MGH_ARNOLDI_SSTEP, 8
        setattr(bad, field, value)
        with pytest.raises(capi.MGHError) as e:
            capi.mgh_workspace_bytes(bad)
        assert e.value.status == capi.MGH_NOT_SUPPORTED, field
    bad = capi.mgh_default_params()
    bad.precision = 3
    with pytest.raises(capi.MGHError):
        capi.mgh_workspace_bytes(bad)


def test_reconstruction_entry_points_validate_on_the_host(lib):
    """mgh_tv_prox / mgh_fbs_momentum reject a missing handle or buffer before any launch."""
    import paper_2107_03679_gb300.capi as capi
    L = capi._lib
    assert L.mgh_tv_prox(None, None, None, 1.0, 0.1, 3, None) == capi.MGH_INVALID_ARG
    assert L.mgh_fbs_momentum(None, None, None, 0.5, None) == capi.MGH_INVALID_ARG
    assert L.mgh_debug_inject_timeout(None) == capi.MGH_INVALID_ARG


@pytest.mark.parametrize("struct", ["mgh_params", "mgh_solve_info", "mgh_profile", "mgh_kernel_shape"])
def test_struct_layouts_match_the_c_header(tmp_path, struct):
    """Each ctypes mirror of a C-ABI struct has the C struct's size and field offsets (compiled
    from include/mgh.h with the host C compiler)."""
    import shutil
    import subprocess
    import paper_2107_03679_gb300.capi as capi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cls = getattr(capi, struct)
    fields = [f for f, _ in cls._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mgh.h"\nint main(void) {\n'
                   f'  printf("%zu\\n", sizeof({struct}));\n'
                   + "".join(f'  printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(cls)
    assert out[1:] == [getattr(cls, f).offset for f in fields]


def test_cycle_type_and_per_level_sweeps_validate_on_the_host(lib):
    import paper_2107_03679_gb300.capi as capi
    p = capi.mgh_default_params()
    base = capi.mgh_workspace_bytes(p)
    p.cycle_type = 2          # the W-cycle keeps one sum of corrections per level 1..L-2
    assert capi.mgh_workspace_bytes(p) > base
    p.cycle_type = 4
    with pytest.raises(capi.MGHError):
        capi.mgh_workspace_bytes(p)
    p.cycle_type = 1
    p.nu_per_level = 1
    for l, (a, b) in enumerate([(2, 1), (1, 0), (0, 3)]):
        p.nu1_level[l], p.nu2_level[l] = a, b
    assert capi.mgh_workspace_bytes(p) == base
    p.nu2_level[1] = 5
    with pytest.raises(capi.MGHError):
        capi.mgh_workspace_bytes(p)
    p.nu2_level[1] = 1
    p.nu1_level[3] = 9        # the coarsest level's entry is ignored
    assert capi.mgh_workspace_bytes(p) == base
    p.nu_per_level = 2
    with pytest.raises(capi.MGHError):
        capi.mgh_workspace_bytes(p)
