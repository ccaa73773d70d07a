"""A plain C program links libqtt.so through include/qtt.h (the header is
valid C) and calls the C-ABI directly: argument validation and host-only
calls on any machine; create / apply / sync / file round trip / destroy
against the C oracle's sweep on a GPU."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "abi_client.c")


def _compile(tmp_path):
    from paper_1511_06029_gb300 import build
    import oracle
    lib = build.build()
    olib = oracle.build()
    cuda = "/usr/local/cuda"
    exe = str(tmp_path / "abi_client")
    cmd = ["gcc", "-std=c11", "-O1", "-Wall", "-Werror", SRC, "-o", exe,
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
           lib, olib, "-L", os.path.join(cuda, "lib64"), "-lcudart", "-lm",
           "-Wl,-rpath," + os.path.dirname(lib), "-Wl,-rpath," + os.path.dirname(olib),
           "-Wl,-rpath," + os.path.join(cuda, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_host(tmp_path):
    exe = _compile(tmp_path)
    r = subprocess.run([exe, "host"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "host ok" in r.stdout, r.stderr


@pytest.mark.gpu
def test_c_client_device(tmp_path):
    exe = _compile(tmp_path)
    r = subprocess.run([exe, "device", str(tmp_path)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and "device ok" in r.stdout, (r.stdout, r.stderr)
