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
