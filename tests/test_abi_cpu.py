"""Host-side checks of the C-ABI library that need no GPU: it loads, exports every
symbol declared in include/afe.h, and validates meshes and parameters on the host."""
import os
import re

import numpy as np
import pytest

from inputs.voronoi import box_voronoi, periodic_voronoi
from oracle.mesh import from_polymesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def afe():
    from paper_2605_00619_gb300 import afe as mod
    if not os.path.exists(mod.LIBPATH):
        from paper_2605_00619_gb300.build import build
        build()
    mod.lib()
    return mod


def test_library_exports_every_declared_symbol(afe):
    header = open(os.path.join(ROOT, "include", "afe.h")).read()
    declared = set(re.findall(r"\b(afe_[a-z_]+)\s*\(", header))
    assert "afe_step" in declared and "afe_mesh_create" in declared
    L = afe.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert declared <= set(afe.exported_symbols())


def test_default_params(afe):
    p = afe.afe_default_params(2)
    assert p.order == 2 and p.gamma == 1.4 and p.R == 1.0 and p.cfl == 0.3 and p.picard_tol == 1e-12
    with pytest.raises(afe.AfeError):
        afe.afe_default_params(5)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_validate_counts_match_oracle(afe, N):
    for pm in (periodic_voronoi(2), box_voronoi(2)):
        p = afe.afe_default_params(N, period=pm.period if pm.periodic else (1, 1, 1))
        bc = afe.AFE_BC_PERIODIC if pm.periodic else afe.AFE_BC_TRANSMISSIVE
        st, nn, nf = afe.afe_mesh_validate(p, pm.xyz, pm.cell_subtet_ptr, pm.subtet_vtx, pm.subtet_shift, bc)
        om = from_polymesh(pm, N)
        assert nn == om.n_nodes
        assert nf == sum(len(c.bfaces) for c in om.cells)


def test_validate_rejects_bad_meshes(afe):
    pm = periodic_voronoi(2)
    p = afe.afe_default_params(1, period=pm.period)
    args = (pm.xyz, pm.cell_subtet_ptr, pm.subtet_vtx, pm.subtet_shift, afe.AFE_BC_PERIODIC)
    assert afe.afe_mesh_validate(p, *args, check=False)[0] == afe.AFE_OK
    # zero-volume sub-tet
    v = pm.subtet_vtx.copy()
    s = pm.subtet_shift.copy()
    v[5, 1], s[5, 1] = v[5, 0], s[5, 0]
    st, _, _ = afe.afe_mesh_validate(p, pm.xyz, pm.cell_subtet_ptr, v, s, afe.AFE_BC_PERIODIC, check=False)
    assert st == afe.AFE_EMESH and "volume" in afe.afe_last_error()
    # a sub-tet missing: the cell is no longer closed and its neighbour's face is unmatched
    keep = np.ones(pm.n_subtets, bool)
    keep[3] = False
    ptr = pm.cell_subtet_ptr.copy()
    ptr[1:] -= 1
    st, _, _ = afe.afe_mesh_validate(p, pm.xyz, ptr, pm.subtet_vtx[keep], pm.subtet_shift[keep],
                                     afe.AFE_BC_PERIODIC, check=False)
    assert st == afe.AFE_EMESH
    # a duplicated sub-tet: non-conforming subgrid
    ptr = pm.cell_subtet_ptr.copy()
    ptr[1:] += 1
    vv = np.insert(pm.subtet_vtx, 0, pm.subtet_vtx[0], axis=0)
    ss = np.insert(pm.subtet_shift, 0, pm.subtet_shift[0], axis=0)
    st, _, _ = afe.afe_mesh_validate(p, pm.xyz, ptr, vv, ss, afe.AFE_BC_PERIODIC, check=False)
    assert st == afe.AFE_EMESH
    # periodic boundary requested for a box mesh: unmatched faces
    bm = box_voronoi(2)
    st, _, _ = afe.afe_mesh_validate(p, bm.xyz, bm.cell_subtet_ptr, bm.subtet_vtx, None, afe.AFE_BC_PERIODIC,
                                     check=False)
    assert st == afe.AFE_EMESH and "unmatched" in afe.afe_last_error()
    # vertex id out of range, bad params
    v = pm.subtet_vtx.copy()
    v[0, 0] = len(pm.xyz) + 3
    assert afe.afe_mesh_validate(p, pm.xyz, pm.cell_subtet_ptr, v, pm.subtet_shift, 0, check=False)[0] != 0
    bad = afe.afe_default_params(1, cfl=-1.0)
    assert afe.afe_mesh_validate(bad, *args, check=False)[0] == afe.AFE_EINVAL


def test_reoriented_subtets_are_accepted(afe):
    pm = box_voronoi(2)
    v = pm.subtet_vtx.copy()
    v[:, [1, 2]] = v[:, [2, 1]]          # every sub-tet negatively oriented
    p = afe.afe_default_params(2)
    st, nn, _ = afe.afe_mesh_validate(p, pm.xyz, pm.cell_subtet_ptr, v, None, afe.AFE_BC_TRANSMISSIVE)
    assert st == afe.AFE_OK and nn == from_polymesh(pm, 2).n_nodes


def test_create_without_gpu_fails_loudly(afe):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    pm = periodic_voronoi(2)
    p = afe.afe_default_params(1, period=pm.period)
    h, st = afe.afe_mesh_create(p, pm.xyz, pm.cell_subtet_ptr, pm.subtet_vtx, pm.subtet_shift, 0, check=False)
    assert h is None and st == afe.AFE_ECUDA


def test_ctypes_structures_match_the_header(tmp_path):
    """Every field of the ctypes mirrors of afe_params and afe_stats sits at the offset the C
    compiler gives it from include/afe.h, and the sizes agree."""
    import ctypes
    import shutil
    import subprocess

    from paper_2605_00619_gb300 import afe as mod
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = []
    for cls in (mod.afe_params, mod.afe_stats):
        name = cls.__name__
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "afe.h"\nint main(void) {\n'
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, field, val = line.split()
            got[(name, field)] = int(val)
    for cls in (mod.afe_params, mod.afe_stats):
        name = cls.__name__
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
