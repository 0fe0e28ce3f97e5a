"""The C ABI from plain C: tests/c/host_abi.c includes include/hytet.h as
C99 (with -pedantic, no warnings allowed), links the built library and runs
its host-only calls without a GPU.  Its output is checked against closed
forms: the unit cube as 6 Kuhn cells has 8 vertices, 19 edges, 18 faces (12
on the boundary), V - E + F - C = 1; t_3(0,2,0) = 5 and t_3(0,0,2) = 9 (the
worked example of the index function, Sec. 4); the quadrature weights sum
to 1; the tile count equals the binding's."""
import os
import shutil
import subprocess

import pytest

import paper_2308_01792_gb300 as hg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    hg.lib()                                     # the library must be built
    libdir = os.path.join(ROOT, "paper_2308_01792_gb300", "lib")
    exe = str(tmp_path_factory.mktemp("c_abi") / "host_abi")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
           "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "host_abi.c"),
           "-L" + libdir, "-lhytet", "-Wl,-rpath," + libdir, "-o", exe]
    p = subprocess.run(cmd, capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    return exe


def test_header_compiles_as_c99_and_host_calls_run(program):
    env = dict(os.environ)
    cuda_lib = "/usr/local/cuda/lib64"
    if os.path.isdir(cuda_lib):
        env["LD_LIBRARY_PATH"] = cuda_lib + os.pathsep + env.get("LD_LIBRARY_PATH", "")
    p = subprocess.run([program], capture_output=True, text=True, env=env, timeout=60)
    assert p.returncode == 0, p.stderr
    lines = p.stdout.strip().splitlines()
    V, E, F, C, Fb, Fi = map(int, lines[0].split()[1:])
    assert (V, E, F, C, Fb, Fi) == (8, 19, 18, 6, 12, 6) and V - E + F - C == 1
    assert lines[1] == "tw3 020 5" and lines[2] == "tw3 002 9"
    assert lines[3] == "tw3 bad -1"                     # HG_ERR_INVALID_ARG outside I_tet(3)
    _, npts, wsum = lines[4].split()
    assert int(npts) == 14 and abs(float(wsum) - 1.0) < 1e-14
    assert lines[5] == f"tiles5 {len(hg.plane_tiles(5))}"
