"""The library from plain C: tests/c_abi_example.c, compiled with the system C
compiler against include/vlbm.h (C99, no C++), linked against the in-tree
libvlbm.so, with no Python or PyTorch in its process.  On the CPU: the header
and the program compile as C.  On the GPU: the program runs a 2-D ideal-MHD
domain through vlbm_create / vlbm_init_fields / vlbm_step / vlbm_moments /
vlbm_conservation / vlbm_destroy and checks exact conservation and the uniform
fixed point itself."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "c_abi_example.c")


def _cc():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    return cc


def test_header_and_example_compile_as_c99(tmp_path):
    obj = tmp_path / "example.o"
    res = subprocess.run([_cc(), "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                          "-I", os.path.join(ROOT, "include"), "-c", SRC, "-o", str(obj)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    assert obj.exists()


@pytest.mark.gpu
def test_example_program_runs_on_the_gpu(tmp_path):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_00641_gb300 import _build
    lib = _build.build()  # the in-tree library (up to date: nothing is recompiled)
    libdir = os.path.dirname(lib)
    exe = tmp_path / "example"
    res = subprocess.run([_cc(), "-std=c99", "-I", os.path.join(ROOT, "include"), SRC, "-o", str(exe),
                          "-L", libdir, "-lvlbm", "-Wl,-rpath," + libdir, "-lm"], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stderr
    assert run.stdout.startswith("c-abi ok"), run.stdout
