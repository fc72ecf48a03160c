"""The step-kernel digest that ties profiles/ traffic figures to the kernel
sources must not depend on where the repository sits (the GPU machine builds
from another directory)."""
import shutil

from paper_2309_04872_gb300 import build as B


def test_step_kernel_digest_is_path_independent(tmp_path, monkeypatch):
    here = B.step_kernel_digest()
    copy = tmp_path / "elsewhere"
    shutil.copytree(B.CSRC, copy / "csrc")
    shutil.copytree(B.INCLUDE, copy / "include")
    flags = [str(copy / "include") if f == B.INCLUDE else f for f in B.NVCC_FLAGS]
    monkeypatch.setattr(B, "CSRC", str(copy / "csrc"))
    monkeypatch.setattr(B, "INCLUDE", str(copy / "include"))
    monkeypatch.setattr(B, "NVCC_FLAGS", flags)
    assert B.step_kernel_digest() == here


def test_step_kernel_digest_follows_the_sources(tmp_path, monkeypatch):
    here = B.step_kernel_digest()
    copy = tmp_path / "csrc"
    shutil.copytree(B.CSRC, copy)
    with open(copy / "lb_step.cuh", "a") as f:
        f.write("\n")
    monkeypatch.setattr(B, "CSRC", str(copy))
    assert B.step_kernel_digest() != here
