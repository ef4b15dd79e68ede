"""The boundary as a C program sees it (no GPU): include/recoil.h compiles as
strict C11 and a C caller links librecoil.so and uses the host-side entry
points (encode under both split rules, combine, export/import, packed
metadata, plan sizes and error codes); see c_abi_check.c."""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_c_caller_uses_the_host_entry_points(recoil_lib, tmp_path):
    lib = recoil_lib.LIB_PATH
    exe = str(tmp_path / "c_abi_check")
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-O1",
           "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "c_abi_check.c"),
           "-L", os.path.dirname(lib), "-l:" + os.path.basename(lib),
           "-Wl,-rpath," + os.path.dirname(lib), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "ok"


def test_header_compiles_as_c99_and_cxx():
    for std, comp in (("c99", "gcc"), ("c++17", "g++")):
        src = "#include \"recoil.h\"\nint main(void) { return RECOIL_OK; }\n"
        cmd = [comp, f"-std={std}", "-Wall", "-Werror", "-pedantic", "-fsyntax-only", "-x",
               "c" if comp == "gcc" else "c++", "-I", os.path.join(ROOT, "include"), "-"]
        r = subprocess.run(cmd, input=src, capture_output=True, text=True)
        assert r.returncode == 0, (std, r.stderr)
