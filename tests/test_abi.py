"""Host-side checks of the C ABI (no GPU needed, no compute call made).

* the shared library loads and exports every function include/p3maze.h declares,
  and exports no p3maze_* function that the header does not declare;
* the ctypes structures have the C layout (sizes and offsets from gcc);
* p3maze_init rejects invalid parameters before it touches the device.
"""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2606_31379_b300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "p3maze.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(p3maze_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    from paper_2606_31379_b300 import p3maze as P
    names = _declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(P.lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", P._LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (p3maze_\w+)", out))
    assert set(names) <= exported
    # and nothing is exported that the header does not declare
    assert exported <= set(names), sorted(exported - set(names))


def test_ctypes_layout_matches_c(tmp_path):
    from paper_2606_31379_b300 import p3maze as P
    structs = {"p3maze_params": P.Params, "p3maze_sr_table": P.SRTable, "p3maze_topology": P.Topology,
               "p3maze_energies": P.Energies, "p3maze_stats": P.Stats, "p3maze_timing": P.Timing, "p3maze_tuning": P.Tuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "p3maze.h"', "int main(void){"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for cname, cls in structs.items():
        import ctypes
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def _base_kwargs(s):
    return dict(alpha=0.30, r_cut=9.0, mesh=32, tol=1e-6, dt=1.0)


@pytest.mark.parametrize("change, needle", [
    (dict(mesh=65), "mesh"),               # odd and above 64, the largest exactly solved level
    (dict(mesh=134), "mesh"),              # 134 -> 67: odd and above 64
    (dict(coarse_max=-1), "coarse_max"),
    (dict(mesh=2), "mesh"),
    (dict(r_cut=30.0), "r_cut"),
    (dict(tol=0.0), "tol"),
    (dict(order=6), "order"),
    (dict(predictor=4), "predictor"),
    (dict(precision="fp64", alpha=-1.0), "alpha"),
    (dict(mesh=8, alpha=0.9), "too coarse"),
    (dict(method="pmaze", alpha=-1.0), "alpha"),
    (dict(method="pmaze", lr_force="analytic"), "finite-difference"),
])
def test_init_rejects_invalid_parameters(change, needle):
    from paper_2606_31379_b300 import p3maze as P
    s = S.nacl_melt(64, 25.2, seed=1)
    kw = _base_kwargs(s)
    kw.update(change)
    with pytest.raises(P.P3MaZeError) as ei:
        P.Context(s.pos, s.charge, s.mass, s.box, vel=s.vel, types=s.types, sr_kind="bmh",
                  sr_table=s.sr_table, **kw)
    assert ei.value.code == P.ERR_INVALID
    assert needle in str(ei.value)


def test_init_rejects_non_neutral_and_bad_types():
    from paper_2606_31379_b300 import p3maze as P
    s = S.nacl_melt(64, 25.2, seed=1)
    q = s.charge.copy()
    q[0] += 0.5
    with pytest.raises(P.P3MaZeError, match="neutral"):
        P.Context(s.pos, q, s.mass, s.box, **_base_kwargs(s))
    t = s.types.copy()
    t[3] = 7
    with pytest.raises(P.P3MaZeError, match="type"):
        P.Context(s.pos, s.charge, s.mass, s.box, types=t, sr_kind="bmh", sr_table=s.sr_table,
                  **_base_kwargs(s))
    w = S.spcfw_water(8, 12.0, seed=1)
    tri = w.angles.copy()
    tri[1, 0] = tri[0, 0]                       # one atom in two molecules
    with pytest.raises(P.P3MaZeError, match="disjoint"):
        P.Context(w.pos, w.charge, w.mass, w.box, types=w.types, sr_kind="lj", sr_table=w.sr_table,
                  triples=tri, bonded=w.bonded, alpha=0.3, r_cut=6.0, mesh=16, tol=1e-6, dt=0.5)
    m = s.mass.copy()
    m[5] = 0.0
    with pytest.raises(P.P3MaZeError, match="mass"):
        P.Context(s.pos, s.charge, m, s.box, **_base_kwargs(s))
    pos = s.pos.copy()
    pos[2, 1] = np.nan
    with pytest.raises(P.P3MaZeError, match="non-finite"):
        P.Context(pos, s.charge, s.mass, s.box, **_base_kwargs(s))


def test_pmaze_rejects_a_molecular_topology_before_touching_the_device():
    from paper_2606_31379_b300 import p3maze as P
    w = S.spcfw_water(8, 12.0, seed=1)
    with pytest.raises(P.P3MaZeError, match="topology") as ei:
        P.Context.from_system(w, alpha=0.0, r_cut=6.0, mesh=16, tol=1e-6, dt=0.5, method="pmaze")
    assert ei.value.code == P.ERR_INVALID
