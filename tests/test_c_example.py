"""The plain-C example (paper_2109_00661_gb300/examples/loglik_c.c) builds
against the C ABI alone (CPU: compile and link), and on a GPU it evaluates the
forward model and the likelihood through it: the unperturbed copy of the
earth that generated the data scores highest."""
import os
import shutil
import subprocess

import pytest

from paper_2109_00661_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2109_00661_gb300", "examples", "loglik_c.c")


def compile_example(out):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    try:
        nvcc = build.nvcc_path()
    except RuntimeError:
        pytest.skip("nvcc not available")
    cuda = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    build.build()
    libdir = os.path.dirname(build.LIB)
    cmd = [cc, "-O2", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"), SRC,
           "-L", libdir, "-laemrjsmc", "-L", os.path.join(cuda, "lib64"), "-lcudart", f"-Wl,-rpath,{libdir}",
           "-lm", "-o", out]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    return out


def test_c_example_builds(tmp_path):
    assert os.path.exists(compile_example(str(tmp_path / "loglik_c")))


@pytest.mark.gpu
def test_c_example_runs(tmp_path):
    exe = compile_example(str(tmp_path / "loglik_c"))
    res = subprocess.run([exe, "2048"], capture_output=True, text=True, timeout=300)
    print(res.stdout)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "best model 0 of 2048" in res.stdout
