"""The ABI from plain C: tests/c/render_one.c compiles against include/vgr.h
and links against libvgr.so here (no GPU needed); where a GPU is present it
also runs and renders its frame."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(tmp_path):
    from paper_2506_02774_gb300 import _build
    lib = _build.build()
    exe = tmp_path / "render_one"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", _build.INCLUDE,
                    os.path.join(ROOT, "tests", "c", "render_one.c"), "-o", str(exe),
                    "-L", os.path.dirname(lib), "-lvgr", "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    return exe


def test_c_client_compiles_and_links(tmp_path):
    assert _build(tmp_path).exists()


@pytest.mark.gpu
def test_c_client_renders(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = subprocess.run([str(_build(tmp_path))], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "cut 2 nodes" in out.stdout
