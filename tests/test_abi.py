"""The C ABI library builds for sm_103a, loads, and exports every declared symbol (no GPU needed)."""
import ctypes
import re
from pathlib import Path

from paper_2511_14955_gb300 import _build, binding

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    text = (ROOT / "include" / "intergrams.h").read_text()
    return sorted(set(re.findall(r"^\s*(?:ig_status|void|const char\*)\s+(intergrams_\w+)\s*\(", text, re.M)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(binding.EXPORTS)


def test_library_builds_loads_and_exports():
    path = _build.build_cuda()
    lib = ctypes.CDLL(str(path))
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_last_error_is_empty_initially():
    lib = binding.load(build_if_missing=False)
    assert lib.intergrams_last_error() == b""


def test_null_arguments_rejected_without_gpu():
    lib = binding.load(build_if_missing=False)
    assert lib.intergrams_plan(None, None, None, 0, None, None, None) == -1
    assert lib.intergrams_pass(None, None) == -1
    assert lib.intergrams_run(None) == -1
    lib.intergrams_free(None)


def struct_fields(name):
    """uint32_t fields of `typedef struct { ... } name;` in the header, in order."""
    text = (ROOT / "include" / "intergrams.h").read_text()
    end = text.index("} " + name + ";")
    body = text[text.rindex("typedef struct {", 0, end):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return re.findall(r"uint32_t\s+(\w+)\s*;", body)


def test_tuning_struct_matches_header():
    """The binding's IgTuning lists the header's ig_tuning fields in order (all uint32_t)."""
    fields = struct_fields("ig_tuning")
    assert [f for f, _ in binding.IgTuning._fields_] == fields
    assert ctypes.sizeof(binding.IgTuning) == 4 * len(fields)


def test_params_struct_matches_header():
    fields = struct_fields("ig_params")
    assert [f for f, _ in binding.IgParams._fields_] == fields


def test_plain_c_program_compiles_links_and_calls(tmp_path):
    """The header is plain C99 (no C++ in it), and a C program that takes the
    address of every declared call links against the library and runs the
    calls that need no GPU."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if not gcc:
        import pytest
        pytest.skip("gcc not available")
    lib = _build.build_cuda()
    names = declared_functions()
    src = tmp_path / "use_abi.c"
    src.write_text(
        "#include <stdio.h>\n#include <string.h>\n#include \"intergrams.h\"\n"
        "typedef void (*fn)(void);\n"
        "int main(void) {\n"
        "  fn table[] = {" + ", ".join(f"(fn){n}" for n in names) + "};\n"
        "  for (size_t i = 0; i < sizeof(table) / sizeof(table[0]); ++i) if (!table[i]) return 2;\n"
        "  if (strcmp(intergrams_last_error(), \"\") != 0) return 3;\n"
        "  if (intergrams_plan(NULL, NULL, NULL, 0, NULL, NULL, NULL) != IG_EINVAL) return 4;\n"
        "  if (intergrams_last_error()[0] == '\\0') return 5;\n"
        "  intergrams_free(NULL);\n"
        "  puts(\"abi ok\");\n"
        "  return 0;\n"
        "}\n")
    exe = tmp_path / "use_abi"
    cuda_lib = "/usr/local/cuda/lib64"
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", str(ROOT / "include"),
           str(src), "-o", str(exe), "-L", str(lib.parent), "-lintergrams", f"-Wl,-rpath,{lib.parent}",
           f"-Wl,-rpath-link,{cuda_lib}", f"-Wl,-rpath,{cuda_lib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "abi ok" in r.stdout, (r.returncode, r.stdout, r.stderr)
