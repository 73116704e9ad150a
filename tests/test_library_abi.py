"""CPU checks of the C ABI: the library builds and loads, exports every symbol include/nqs.h
declares, and its host-side validation and parameter layout behave (no device work here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_2208_05637_b300 as P
    return P


def _declared():
    text = open(os.path.join(ROOT, "include", "nqs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nqs_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(so, n), n
    assert sorted(lib.EXPORTED) == names


def test_status_strings(lib):
    for code in range(0, -10, -1):
        assert lib._lib.nqs_strerror(code)


def test_ham_create_validation_errors(lib):
    import ctypes
    m = np.zeros(3, dtype=np.uint64)
    c = np.ones(1)
    h = ctypes.c_void_p()
    # more than 128 qubits (three words) is out of range
    assert lib._lib.nqs_ham_create(129, 1, m.ctypes.data_as(ctypes.c_void_p), m.ctypes.data_as(ctypes.c_void_p),
                                   c.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)) == lib.NQS_ERR_NQUBITS
    with pytest.raises(ValueError):
        lib.Hamiltonian(65, [0], [0], [1.0])          # 65 qubits need [K, 2] masks
    with pytest.raises(lib.NQSError) as e:
        lib.Hamiltonian(66, [[0, 1 << 2]], [[0, 0]], [1.0])   # qubit 66 of a 66-qubit register
    assert e.value.status == lib.NQS_ERR_INVALID_ARG
    with pytest.raises(lib.NQSError) as e:
        lib.Hamiltonian(4, [1 << 4], [0], [1.0])
    assert e.value.status == lib.NQS_ERR_INVALID_ARG
    with pytest.raises(lib.NQSError) as e:
        lib.Hamiltonian(4, [1], [0], [float("nan")])
    assert e.value.status == lib.NQS_ERR_NAN


def test_model_create_validation_errors(lib):
    with pytest.raises(lib.NQSError) as e:
        lib.Model("made", 3, 1, 1, 16, 1)
    assert e.value.status == lib.NQS_ERR_NQUBITS
    with pytest.raises(lib.NQSError) as e:
        lib.Model("made", 8, 5, 1, 16, 1)
    assert e.value.status == lib.NQS_ERR_INVALID_ARG
    with pytest.raises(lib.NQSError) as e:
        lib.Model("made", 8, 1, 1, 16, 1, order=[0, 0, 1, 2, 3, 4, 5, 6])
    assert e.value.status == lib.NQS_ERR_INVALID_ARG
    with pytest.raises(lib.NQSError) as e:
        lib.Model("transformer", 8, 1, 1, 48, 2, 2)   # head size 24
    assert e.value.status == lib.NQS_ERR_UNSUPPORTED


@pytest.mark.parametrize("arch,n,h,l,heads", [("made", 12, 64, 2, 0), ("made", 4, 16, 1, 0),
                                              ("product", 20, 0, 0, 0),
                                              ("transformer", 20, 64, 2, 4),
                                              ("transformer", 52, 128, 4, 8)])
def test_param_layout_matches_named_shapes(lib, arch, n, h, l, heads):
    m = lib.Model(arch, n, 2, 2, h, l, heads)
    layout = m.param_layout()
    shapes = synth.param_shapes(arch, n, h, l, heads)
    assert [x[0] for x in layout] == [s[0] for s in shapes]
    off = 0
    for (name, o, numel), (_, shape) in zip(layout, shapes):
        assert o == off and numel == int(np.prod(shape)), name
        off += numel
    assert m.param_count == off
    params = synth.init_params(arch, n, 2, 2, h, l, heads, seed=1)
    flat = np.concatenate([params[s[0]].ravel() for s in shapes])
    back = m.unpack(flat)
    for k, v in params.items():
        assert np.array_equal(back[k], v.ravel())


def test_workspace_sizes_grow_with_batch(lib):
    m = lib.Model("made", 12, 2, 2, 64, 2)
    a = ctypes.c_size_t(); b = ctypes.c_size_t()
    assert lib._lib.nqs_workspace_size(m.handle, None, lib.OP_BACKWARD, 10, ctypes.byref(a)) == 0
    assert lib._lib.nqs_workspace_size(m.handle, None, lib.OP_BACKWARD, 1000, ctypes.byref(b)) == 0
    assert b.value > a.value
    assert lib._lib.nqs_workspace_size(m.handle, None, lib.OP_LOCAL_ENERGY, 10, ctypes.byref(a)) == lib.NQS_ERR_INVALID_ARG


def test_package_has_no_cpu_fallback():
    src = open(os.path.join(ROOT, "paper_2208_05637_b300", "__init__.py")).read()
    assert "raise ImportError" in src
    for p in ("__init__.py", "vmc.py"):
        body = open(os.path.join(ROOT, "paper_2208_05637_b300", p)).read()
        assert "import oracle" not in body and "from oracle" not in body
