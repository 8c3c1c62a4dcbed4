"""The C ABI library loads and exports every symbol include/dh2.h declares (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dh2.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dh2_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1809_04384_gb300.build import build

    return build()


def test_header_declares_boundary():
    names = _declared()
    for required in ("dh2_build_tree", "dh2_build_dh2", "dh2_matvec", "dh2_matvec_host", "dh2_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (dh2_[a-z0-9_]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binds(libpath):
    import paper_1809_04384_gb300 as pkg

    L = pkg.lib()
    for name in _declared():
        assert hasattr(L, name)
    # binding covers the same names
    assert sorted(pkg.exported_symbols()) == _declared()
    # host-only entry points work without a GPU
    o = pkg.options()
    assert o.eta1 == 10.0 and o.leaf_max == 32 and o.precision == pkg.DH2_MIXED
    assert pkg.lib().dh2_stage_name(0) == b"structure"
    assert pkg.lib().dh2_stage_name(99) is None


def test_invalid_arguments_rejected_before_gpu_work(libpath):
    import ctypes as C

    import numpy as np

    import paper_1809_04384_gb300 as pkg

    with pytest.raises(pkg.DH2Error) as e:
        pkg.dh2_build_tree(np.zeros((0, 3)), None)
    assert e.value.status == pkg.DH2_EINVAL
    v = np.eye(3)
    with pytest.raises(pkg.DH2Error) as e:
        pkg.dh2_build_tree(v, np.array([[0, 1, 5]]))
    assert e.value.status == pkg.DH2_EINVAL
    with pytest.raises(pkg.DH2Error) as e:
        pkg.dh2_build_dh2(None, 1.0, 4, 1.0, 1e-4)
    assert e.value.status == pkg.DH2_EINVAL
    # dh2_gram: NULL pointers, sizes and the mode are checked before any device work
    L = pkg.lib()
    buf = (C.c_double * 4)()
    assert L.dh2_gram(None, 8, 4, 4, 1, buf, None) == pkg.DH2_EINVAL
    assert L.dh2_gram(buf, 8, 4, 4, 1, None, None) == pkg.DH2_EINVAL
    assert L.dh2_gram(buf, 0, 4, 4, 1, buf, None) == pkg.DH2_EINVAL
    assert L.dh2_gram(buf, 8, 513, 513, 1, buf, None) == pkg.DH2_EINVAL
    assert L.dh2_gram(buf, 8, 4, 3, 1, buf, None) == pkg.DH2_EINVAL
    assert L.dh2_gram(buf, 8, 4, 4, 2, buf, None) == pkg.DH2_EINVAL
    # the option defaults to the tensor-core Gram and takes only 0 / 1
    assert pkg.options().gram_tc == 1


def test_batch_arguments_rejected_before_gpu_work(libpath):
    import ctypes as C

    import paper_1809_04384_gb300 as pkg

    L = pkg.lib()
    assert L.dh2_build_dh2_batch(None, -1, None, 5, 1.0, 1e-4, None, 0, None) == pkg.DH2_EINVAL
    assert L.dh2_build_dh2_batch(None, 2, None, 5, 1.0, 1e-4, None, 0, None) == pkg.DH2_EINVAL
    # a NULL tree inside the batch: every output slot is cleared, nothing is built
    trees = (C.c_void_p * 2)(None, None)
    kappas = (C.c_double * 2)(1.0, 2.0)
    out = (C.c_void_p * 2)(1, 1)
    st = L.dh2_build_dh2_batch(C.cast(trees, C.c_void_p), 2, C.cast(kappas, C.c_void_p), 5, 1.0, 1e-4, None, 0,
                               C.cast(out, C.c_void_p))
    assert st == pkg.DH2_EINVAL and out[0] is None and out[1] is None
    assert b"tree is NULL" in L.dh2_last_error()
    assert L.dh2_build_dh2_batch(None, 0, None, 5, 1.0, 1e-4, None, -1, None) == pkg.DH2_EINVAL
    assert L.dh2_build_dh2_batch(None, 0, None, 5, 1.0, 1e-4, None, 0, None) == pkg.DH2_OK
    assert L.dh2_matvec_batch(None, 1, None, None, pkg.DH2_C64, None) == pkg.DH2_EINVAL
    mats = (C.c_void_p * 1)(None)
    xs = (C.c_void_p * 1)(None)
    assert L.dh2_matvec_batch(C.cast(mats, C.c_void_p), 1, C.cast(xs, C.c_void_p), C.cast(xs, C.c_void_p),
                              pkg.DH2_C64, None) == pkg.DH2_EINVAL
    assert L.dh2_matvec_batch(None, 0, None, None, 7, None) == pkg.DH2_EINVAL
    assert L.dh2_matvec_batch(None, 0, None, None, pkg.DH2_C64, None) == pkg.DH2_OK


def test_struct_layouts_match_header(libpath, tmp_path):
    """The ctypes mirrors of dh2_options / dh2_matrix_info have the C sizes and offsets."""
    import ctypes as C

    import paper_1809_04384_gb300 as pkg

    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "dh2.h"\n'
        "int main(void) {\n"
        '  printf("%zu %zu %zu %zu %zu\\n", sizeof(dh2_options), offsetof(dh2_options, model),\n'
        "         sizeof(dh2_matrix_info), offsetof(dh2_matrix_info, learned_m),\n"
        "         offsetof(dh2_matrix_info, truncation_bytes));\n  return 0;\n}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [C.sizeof(pkg.dh2_options), pkg.dh2_options.model.offset, C.sizeof(pkg.dh2_matrix_info),
            pkg.dh2_matrix_info.learned_m.offset, pkg.dh2_matrix_info.truncation_bytes.offset]
    assert got == want


def test_learned_arguments_rejected_before_gpu_work(libpath):
    import ctypes as C

    import numpy as np

    import paper_1809_04384_gb300 as pkg

    L = pkg.lib()
    o = pkg.options()
    assert o.learned == 0 and not o.model
    h = C.c_void_p()
    assert L.dh2_model_create(None, None, C.byref(h)) == pkg.DH2_EINVAL and not h.value
    p = np.zeros(pkg.DH2_MLP_NPARAMS, dtype=np.float32)
    p[17] = np.nan
    assert L.dh2_model_create(C.c_void_p(p.ctypes.data), None, C.byref(h)) == pkg.DH2_EINVAL
    assert b"non-finite" in L.dh2_last_error()
    assert L.dh2_model_forward(None, None, 4, None, None) == pkg.DH2_EINVAL
    assert L.dh2_model_grad(None, None, None, 4, None, None, None) == pkg.DH2_EINVAL
    assert L.dh2_model_train_step(None, None, None, 4, 1e-3, None, None) == pkg.DH2_EINVAL
    n = C.c_int64(-1)
    assert L.dh2_learned_features(None, 1.0, 1.0, None, None, None, 0, C.byref(n), None) == pkg.DH2_EINVAL
    assert L.dh2_learned_probe(None, 1.0, 1.0, None, None, None, 0, C.byref(n)) == pkg.DH2_EINVAL
    assert L.dh2_learned_features(None, 1.0, 1.0, None, None, None, 0, None, None) == pkg.DH2_EINVAL
    # a learned build without a model
    o.learned = 1
    assert L.dh2_build_dh2(None, 1.0, 5, 1.0, 1e-4, C.byref(o), None, C.byref(h)) == pkg.DH2_EINVAL


def test_autotune_arguments_rejected_before_gpu_work(libpath):
    import ctypes as C

    import paper_1809_04384_gb300 as pkg

    L = pkg.lib()
    o = pkg.options()
    assert list(o.qr_tpc) == [0, 0, 0]
    t = pkg.dh2_options()
    assert L.dh2_autotune(None, 1.0, 5, 1.0, 1e-4, C.byref(o), 1, None, C.byref(t), None, None) == pkg.DH2_EINVAL
    assert L.dh2_autotune(None, 1.0, 5, 1.0, 1e-4, C.byref(o), 0, None, C.byref(t), None, None) == pkg.DH2_EINVAL
    assert L.dh2_autotune(None, 1.0, 5, 1.0, 1e-4, C.byref(o), 1, None, None, None, None) == pkg.DH2_EINVAL


def test_null_handles_rejected_before_gpu_work(libpath):
    """Every entry point that takes a handle refuses a NULL one with DH2_EINVAL and a message,
    without touching the device."""
    import ctypes as C

    import paper_1809_04384_gb300 as pkg

    L = pkg.lib()
    i32 = C.c_int32()
    buf = (C.c_double * 16)()
    calls = {
        "dh2_matvec": lambda: L.dh2_matvec(None, buf, buf, pkg.DH2_C64, None),
        "dh2_matvec_noalloc": lambda: L.dh2_matvec_noalloc(None, buf, buf, pkg.DH2_C64, None),
        "dh2_matvec_host": lambda: L.dh2_matvec_host(None, buf, buf, None),
        "dh2_set_timing": lambda: L.dh2_set_timing(None, 1),
        "dh2_tree_get_info": lambda: L.dh2_tree_get_info(None, C.byref(pkg.dh2_tree_info())),
        "dh2_tree_export": lambda: L.dh2_tree_export(None, *([None] * 9)),
        "dh2_matrix_get_info": lambda: L.dh2_matrix_get_info(None, C.byref(pkg.dh2_matrix_info())),
        "dh2_export_directions": lambda: L.dh2_export_directions(None, 0, C.byref(i32), None, None, None),
        "dh2_export_blocks": lambda: L.dh2_export_blocks(None, None, None, None),
        "dh2_export_pair": lambda: L.dh2_export_pair(None, 0, 0, buf, 16, C.byref(i32), C.byref(i32)),
        "dh2_export_ranks": lambda: L.dh2_export_ranks(None, None, None),
        "dh2_dense_rows": lambda: L.dh2_dense_rows(None, 1.0, None, 1, None, None, None),
        "dh2_model_get_params": lambda: L.dh2_model_get_params(None, None),
    }
    for name, call in calls.items():
        assert call() == pkg.DH2_EINVAL, name
        assert L.dh2_last_error(), name
    # freeing NULL handles is a no-op
    L.dh2_free_tree(None)
    L.dh2_free_matrix(None)
    L.dh2_free_model(None)
