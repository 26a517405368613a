"""The C-ABI library builds, loads without a GPU and exports every entry point that
include/fc.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fc_[a-z_0-9]+)\s*\(", src))
    return names


def test_library_exports_declared_symbols():
    from paper_1809_01971_gb300 import build, fc
    if not os.path.exists(fc.LIB_PATH):
        build.build()
    lib = ctypes.CDLL(fc.LIB_PATH)
    names = _declared()
    assert {"fc_setup", "fc_apply", "fc_precond", "fc_truncate", "fc_solve", "fc_inner"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    # every declared name is bound by the Python binding with the same name
    fc.lib()
    assert all(hasattr(fc.lib(), n) for n in names)


def test_strerror_is_host_only():
    from paper_1809_01971_gb300 import fc
    L = fc.lib()
    assert L.fc_strerror(fc.FC_ERANK).decode() == "rank capacity exceeded"
    assert L.fc_strerror(12345).decode() == "unknown error"


def test_setup_rejects_bad_parameters_without_touching_the_gpu():
    """Argument checks run before any CUDA call (paper range 0 < alpha <= 1, d in {2,3})."""
    from paper_1809_01971_gb300 import fc
    L = fc.lib()
    out = ctypes.c_void_p()
    for args in [(63, 4, 0.5, 1.0, 1e-2, 1e-8), (63, 2, 1.5, 1.0, 1e-2, 1e-8),
                 (0, 2, 0.5, 1.0, 1e-2, 1e-8), (63, 2, 0.5, -1.0, 1e-2, 1e-8),
                 (63, 3, 0.5, 1.0, 0.0, 1e-8), (63, 3, 0.5, 1.0, 1e-2, 0.0)]:
        assert L.fc_setup(*args, None, ctypes.byref(out)) == fc.FC_EINVAL


def test_import_sets_work_queues_unless_the_caller_did():
    """Importing the package asks CUDA for 32 hardware work queues, so that the streams of a
    batched solve do not serialise behind each other, and keeps a value the caller set."""
    import subprocess
    import sys
    code = ("import os, sys; sys.path.insert(0, {root!r}); import paper_1809_01971_gb300; "
            "print(os.environ['CUDA_DEVICE_MAX_CONNECTIONS'])").format(root=ROOT)
    env = {k: v for k, v in os.environ.items() if k != "CUDA_DEVICE_MAX_CONNECTIONS"}
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "32"
    env["CUDA_DEVICE_MAX_CONNECTIONS"] = "4"
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "4"


def test_header_is_plain_c_and_links_from_c(tmp_path):
    """include/fc.h compiles as pedantic C99 and a C program links against libfc.so and gets
    the host-only answers (argument errors, status strings) without a GPU."""
    import shutil
    import subprocess
    from paper_1809_01971_gb300 import fc
    gcc = shutil.which("gcc")
    if gcc is None:
        import pytest
        pytest.skip("gcc not available")
    fc.lib()                                     # built in-tree
    libdir = os.path.dirname(fc.LIB_PATH)
    exe = str(tmp_path / "abi_from_c")
    subprocess.run([gcc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_from_c.c"), "-o", exe,
                    "-L", libdir, "-lfc", "-Wl,-rpath," + libdir],
                   check=True, capture_output=True, timeout=300)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "ok"


def test_binding_has_every_entry_point_by_name():
    """The Python binding exposes each C entry point under the same name; the host-only ones
    answer without a GPU."""
    import paper_1809_01971_gb300 as pkg
    from paper_1809_01971_gb300 import fc
    missing = [n for n in sorted(_declared()) if not hasattr(pkg, n)]
    assert not missing, missing
    assert pkg.fc_strerror(fc.FC_ERANK) == "rank capacity exceeded"
    assert pkg.fc_strerror(fc.FC_ETIMEOUT).startswith("a bounded wait")
    assert isinstance(pkg.fc_last_cuda_error(), str)
