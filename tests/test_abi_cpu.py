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
    assert afe.afe_default_params(4).order == 4
    with pytest.raises(afe.AfeError):
        afe.afe_default_params(5)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
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
    for cls in (mod.afe_params, mod.afe_stats, mod.afe_plan, mod.afe_schedule):
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
    for cls in (mod.afe_params, mod.afe_stats, mod.afe_plan, mod.afe_schedule):
        name = cls.__name__
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


_C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "afe.h"

/* one cube [0,1]^3 split into 24 fan sub-tets: corners 0-7 (bit i of the id = coordinate
   i), the centre 8, face centres 9-14 */
int main(void) {
  double xyz[15 * 3];
  for (int v = 0; v < 8; ++v)
    for (int d = 0; d < 3; ++d) xyz[v * 3 + d] = (v >> d) & 1;
  for (int d = 0; d < 3; ++d) xyz[8 * 3 + d] = 0.5;
  int64_t vtx[24 * 4];
  int k = 0, f = 9;
  for (int ax = 0; ax < 3; ++ax)
    for (int side = 0; side < 2; ++side, ++f) {
      int e1 = (ax + 1) % 3, e2 = (ax + 2) % 3;
      for (int d = 0; d < 3; ++d) xyz[f * 3 + d] = d == ax ? side : 0.5;
      int ring[4], uv[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
      for (int r = 0; r < 4; ++r) ring[r] = (side << ax) | (uv[r][0] << e1) | (uv[r][1] << e2);
      for (int r = 0; r < 4; ++r, ++k) {
        vtx[k * 4 + 0] = 8;
        vtx[k * 4 + 1] = f;
        vtx[k * 4 + 2] = ring[r];
        vtx[k * 4 + 3] = ring[(r + 1) % 4];
      }
    }
  int64_t ptr[2] = {0, 24};
  afe_params p;
  if (afe_default_params(&p, 2) != AFE_OK) return 1;
  int64_t nodes = -1, tris = -1;
  int st = afe_mesh_validate(&p, 15, xyz, 1, ptr, vtx, NULL, AFE_BC_TRANSMISSIVE, &nodes, &tris);
  printf("%d %lld %lld\n", st, (long long)nodes, (long long)tris);
  vtx[5] = vtx[4]; /* sub-tet 1: two equal vertices, zero volume */
  st = afe_mesh_validate(&p, 15, xyz, 1, ptr, vtx, NULL, AFE_BC_TRANSMISSIVE, &nodes, &tris);
  printf("%d %s\n", st, afe_last_error());
  st = afe_default_params(&p, 7);
  printf("%d %s\n", st, afe_last_error());
  return 0;
}
"""


def test_c_program_uses_the_abi(afe, tmp_path):
    """A C program built against include/afe.h and linked to the library: default parameters,
    validation of a one-cube mesh (P2 fan subgrid: 15 vertices + 50 subgrid edges = 65 nodes,
    24 boundary sub-triangles), and the error path with its message."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text(_C_PROGRAM)
    exe = tmp_path / "use"
    lib = afe.LIBPATH
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), lib,
                    "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    assert out[0].split() == [str(afe.AFE_OK), "65", "24"]
    assert out[1].startswith(str(afe.AFE_EMESH)) and "volume" in out[1]
    assert out[2].startswith(str(afe.AFE_EINVAL)) and "order" in out[2]
