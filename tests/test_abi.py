"""C ABI checks that need no GPU: the library loads, exports every function
include/ssamg.h declares, and rejects invalid input before touching CUDA."""
import ctypes

import numpy as np
import pytest


def test_exports_every_declared_function(ssamg_lib):
    S = ssamg_lib
    names = S.header_functions()
    assert len(names) >= 25
    L = S.lib()
    for n in names:
        assert hasattr(L, n), n
        assert n in S._SIGS, f"binding lacks a signature for {n}"


def test_fastdiv_constants(ssamg_lib):
    assert ssamg_lib.lib().ssamg_selftest_fastdiv(12345, 500000) == 0
    assert ssamg_lib.lib().ssamg_selftest_fastdiv(99, 500000) == 0


def test_status_strings(ssamg_lib):
    S = ssamg_lib
    for c in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert len(S.status_string(c)) >= 2 and S.status_string(c) != "unknown status"


def _grid(S, ndim, boxes):
    L = S.lib()
    h = ctypes.c_void_p()
    assert L.ssamg_grid_create(ndim, len(boxes), ctypes.byref(h)) == 0
    rcs = [L.ssamg_grid_set_box(h, p, S._ints(lo), S._ints(hi)) for p, (lo, hi) in enumerate(boxes)]
    return h, rcs


def test_grid_validation(ssamg_lib):
    S = ssamg_lib
    L = S.lib()
    h = ctypes.c_void_p()
    assert L.ssamg_grid_create(4, 1, ctypes.byref(h)) == S.ERR_ARG
    assert L.ssamg_grid_create(3, 0, ctypes.byref(h)) == S.ERR_ARG
    g, rcs = _grid(S, 2, [((0, 0, 0), (3, 3, 0)), ((0, 0, 0), (3, 3, 1))])
    assert rcs == [0, S.ERR_ARG]          # unused dimension must be flat
    assert L.ssamg_grid_set_box(g, 1, S._ints((2, 0, 0)), S._ints((1, 3, 0))) == S.ERR_ARG
    assert L.ssamg_grid_assemble(g) == S.ERR_ARG   # part 1 has no box
    assert L.ssamg_grid_num_cells(g) == -1
    assert L.ssamg_grid_set_box(g, 1, S._ints((-2, 0, 0)), S._ints((1, 3, 0))) == 0
    assert L.ssamg_grid_assemble(g) == 0
    assert L.ssamg_grid_num_cells(g) == 16 + 16
    assert L.ssamg_grid_set_box(g, 0, S._ints((0, 0, 0)), S._ints((1, 1, 0))) == S.ERR_STATE
    L.ssamg_grid_destroy(g)


def test_matrix_and_coupling_validation(ssamg_lib):
    S = ssamg_lib
    L = S.lib()
    g, _ = _grid(S, 3, [((0, 0, 0), (3, 3, 3)), ((0, 0, 0), (3, 3, 3))])
    assert L.ssamg_grid_assemble(g) == 0
    A = ctypes.c_void_p()
    assert L.ssamg_matrix_create(g, 2, S._ints([0, 0, 0, 2, 0, 0]), ctypes.byref(A)) == S.ERR_ARG
    assert L.ssamg_matrix_create(g, 2, S._ints([0, 0, 0, 0, 0, 0]), ctypes.byref(A)) == S.ERR_ARG
    offs = [0, 0, 0, 1, 0, 0, -1, 0, 0]
    assert L.ssamg_matrix_create(g, 3, S._ints(offs), ctypes.byref(A)) == 0
    assert L.ssamg_matrix_set_constant(A, 2, 0, 1.0) == S.ERR_ARG
    assert L.ssamg_matrix_set_constant(A, 0, 3, 1.0) == S.ERR_ARG

    def add(part, idx, d, q, nidx):
        v = np.array([-1.0])
        return L.ssamg_matrix_add_couplings(A, 1, S._ints([part]), S._ints(idx), S._ints(d),
                                            S._ints([q]), S._ints(nidx),
                                            v.ctypes.data_as(S._dp))
    assert add(0, (3, 1, 1), (1, 0, 0), 1, (0, 1, 1)) == 0
    assert add(0, (2, 1, 1), (1, 0, 0), 1, (0, 1, 1)) == S.ERR_ARG   # leaves through +x, not on that face
    assert add(0, (2, 1, 1), (0, 0, 0), 1, (0, 1, 1)) == 0            # a non-geometric row may lie inside
    assert add(0, (3, 1, 1), (1, 0, 0), 0, (0, 1, 1)) == S.ERR_ARG   # same part
    assert add(0, (0, 1, 1), (1, 0, 0), 1, (0, 1, 1)) == S.ERR_ARG   # dir leaves through +x but cell is at lo
    assert add(0, (3, 1, 1), (1, 0, 0), 1, (4, 1, 1)) == S.ERR_ARG   # column outside its box
    # every entry of every part needs a value before assembly (no CUDA call yet)
    assert L.ssamg_matrix_assemble(A, None) == S.ERR_ARG
    L.ssamg_matrix_destroy(A)
    L.ssamg_grid_destroy(g)


def test_large_coupling_calls_split_over_threads(ssamg_lib):
    """A call of many couplings is converted in chunks on host threads: a
    valid call is accepted whole, one invalid coupling deep inside a large
    call rejects all of it, and the matrix takes later calls as before."""
    S = ssamg_lib
    L = S.lib()
    g, _ = _grid(S, 3, [((0, 0, 0), (15, 15, 15)), ((16, 0, 0), (31, 15, 15))])
    assert L.ssamg_grid_assemble(g) == 0
    A = ctypes.c_void_p()
    offs = [0, 0, 0, 1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1]
    assert L.ssamg_matrix_create(g, 7, S._ints(offs), ctypes.byref(A)) == 0
    # the +x face of part 0 against the -x face of part 1, repeated (repeats
    # are summed at assembly): 40,960 couplings
    j, k = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    face = np.stack([np.full(256, 15), j.ravel(), k.ravel()], 1)
    idx = np.tile(face, (160, 1)).astype(np.int32)
    n = len(idx)
    nidx = idx.copy()
    nidx[:, 0] = 16
    part = np.zeros(n, np.int32)
    nbor = np.ones(n, np.int32)
    d = np.tile(np.array([[1, 0, 0]], np.int32), (n, 1))
    v = np.full(n, -0.25)

    def add(idx_, d_):
        return L.ssamg_matrix_add_couplings(
            A, n, S._ints(part), S._ints(idx_.ravel()), S._ints(d_.ravel()), S._ints(nbor),
            S._ints(nidx.ravel()), v.ctypes.data_as(S._dp))
    assert add(idx, d) == 0
    bad = idx.copy()
    bad[n - 900, 0] = 14  # leaves through +x but is not on that face
    assert add(bad, d) == S.ERR_ARG
    bad_dir = d.copy()
    bad_dir[7] = (2, 0, 0)  # direction components are -1, 0 or 1
    assert add(idx, bad_dir) == S.ERR_ARG
    assert add(idx, d) == 0
    L.ssamg_matrix_destroy(A)
    L.ssamg_grid_destroy(g)


def test_solver_state_errors(ssamg_lib):
    S = ssamg_lib
    L = S.lib()
    p = S.default_params()
    assert p.tol == 1e-8 and p.max_levels == 64 and p.coarse_direct == 1
    h = ctypes.c_void_p()
    bad = S.default_params(precision=2)
    assert L.ssamg_solver_create(ctypes.byref(bad), ctypes.byref(h)) == S.ERR_ARG
    assert p.rhs_together == 1
    bad = S.default_params(rhs_together=2)
    assert L.ssamg_solver_create(ctypes.byref(bad), ctypes.byref(h)) == S.ERR_ARG
    assert L.ssamg_solver_create(ctypes.byref(p), ctypes.byref(h)) == 0
    x = ctypes.c_void_p(16)
    assert L.ssamg_solve(h, x, x, 1, 1, None, None) == S.ERR_STATE
    assert L.ssamg_num_levels(h) == S.ERR_STATE
    g, _ = _grid(S, 3, [((0, 0, 0), (1, 1, 1))])
    assert L.ssamg_grid_assemble(g) == 0
    A = ctypes.c_void_p()
    assert L.ssamg_matrix_create(g, 1, S._ints([0, 0, 0]), ctypes.byref(A)) == 0
    assert L.ssamg_setup(h, A, None) == S.ERR_STATE     # matrix not assembled
    L.ssamg_solver_destroy(h)
    L.ssamg_matrix_destroy(A)
    L.ssamg_grid_destroy(g)


def test_tile_table_validation(ssamg_lib):
    """The tile table is host state: valid tables round-trip, an invalid
    entry is rejected and leaves the table as it was, NULL restores the
    built-in rule, and the calls that need a hierarchy refuse before setup."""
    S = ssamg_lib
    L = S.lib()
    p = S.default_params()
    h = ctypes.c_void_p()
    assert L.ssamg_solver_create(ctypes.byref(p), ctypes.byref(h)) == 0
    n = S.TILE_CLASSES
    got = (ctypes.c_int * n)()
    assert L.ssamg_get_tile_table(h, got) == 0 and list(got) == [0] * n
    table = [(c % 4 + 1) | (S.TILE_BRICKS if c % 3 == 0 else 0) if c % 5 else 0 for c in range(n)]
    assert L.ssamg_set_tile_table(h, S._ints(table)) == 0
    assert L.ssamg_get_tile_table(h, got) == 0 and list(got) == table
    for bad in (5, -1, S.TILE_BRICKS, S.TILE_BRICKS | 5, 16, 1 | 16):
        t2 = list(table)
        t2[7] = bad
        assert L.ssamg_set_tile_table(h, S._ints(t2)) == S.ERR_ARG, bad
        assert L.ssamg_get_tile_table(h, got) == 0 and list(got) == table
    assert L.ssamg_set_tile_table(h, None) == 0
    assert L.ssamg_get_tile_table(h, got) == 0 and list(got) == [0] * n
    k, b = ctypes.c_int(), ctypes.c_int()
    assert L.ssamg_level_tile(h, 0, ctypes.byref(k), ctypes.byref(b)) == S.ERR_STATE
    assert L.ssamg_autotune(h, 10, None, got) == S.ERR_STATE
    assert L.ssamg_autotune(h, 0, None, got) == S.ERR_ARG
    assert L.ssamg_get_tile_table(None, got) == S.ERR_ARG
    L.ssamg_solver_destroy(h)


def test_binding_constants_match_the_header(ssamg_lib):
    """The binding's copies of the header's constants (status codes, tile
    table size and bit) are the header's values."""
    import re
    S = ssamg_lib
    txt = open(S.HEADER).read()
    defines = dict(re.findall(r"#define\s+(SSAMG_\w+)\s+(-?\d+)", txt))
    assert int(defines["SSAMG_TILE_CLASSES"]) == S.TILE_CLASSES
    assert int(defines["SSAMG_TILE_BRICKS"]) == S.TILE_BRICKS
    codes = dict(re.findall(r"(SSAMG_(?:OK|NOT_CONVERGED|ERR_\w+))\s*=\s*(-?\d+)", txt))
    for name, value in codes.items():
        assert getattr(S, name[len("SSAMG_"):]) == int(value), name


def _header_struct(txt, name):
    """(type, field) pairs of `typedef struct { ... } name;` in the header,
    comments removed."""
    import re
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", txt).group(1)
    fields = []
    for decl in body.split(";"):
        words = decl.split()
        if words:
            fields.append((" ".join(words[:-1]), words[-1]))
    return fields


def test_binding_structs_match_the_header(ssamg_lib):
    """The ctypes copies of ssamg_params and ssamg_stats have the header's
    fields in the header's order and with its C types (a field added on one
    side only would shift every later one)."""
    import ctypes as C
    S = ssamg_lib
    txt = open(S.HEADER).read()
    ctype = {"int": C.c_int, "double": C.c_double, "long long": C.c_longlong}
    for name, cls in (("ssamg_params", S.Params), ("ssamg_stats", S.Stats)):
        want = _header_struct(txt, name)
        got = [(f, t) for f, t in cls._fields_]
        assert [f for _, f in want] == [f for f, _ in got], name
        for (ct, f), (_, t) in zip(want, got):
            assert ctype[ct] is t, (name, f)


def test_binding_errors_without_a_hierarchy(ssamg_lib):
    """The binding raises SsamgError with the library's status for bad
    parameters, bad tile tables and calls that need a set-up hierarchy."""
    S = ssamg_lib
    with pytest.raises(S.SsamgError) as e:
        S.Solver(precision=2)
    assert e.value.code == S.ERR_ARG
    sv = S.Solver()
    assert sv.tile_table() == [0] * S.TILE_CLASSES
    with pytest.raises(S.SsamgError) as e:
        sv.set_tile_table([5] * S.TILE_CLASSES)
    assert e.value.code == S.ERR_ARG
    sv.set_tile_table([2 | S.TILE_BRICKS] * S.TILE_CLASSES)
    assert sv.tile_table() == [2 | S.TILE_BRICKS] * S.TILE_CLASSES
    sv.set_tile_table(None)
    assert sv.tile_table() == [0] * S.TILE_CLASSES
    for call in (lambda: sv.num_levels(), lambda: sv.level_tile(0), lambda: sv.autotune(reps=1)):
        with pytest.raises(S.SsamgError) as e:
            call()
        assert e.value.code == S.ERR_STATE


class _FakeDeviceTensor:
    """Stands in for a CUDA tensor (no GPU needed): the binding's checks read
    only these attributes before any pointer reaches the library."""

    def __init__(self, n, dtype="torch.float64", contiguous=True):
        self.n, self.dtype, self.contig, self.is_cuda = n, dtype, contiguous, True

    def is_contiguous(self):
        return self.contig

    def numel(self):
        return self.n

    def data_ptr(self):
        return 0x1000


def test_binding_checks_device_vectors_before_the_call(ssamg_lib):
    """A device vector of the wrong dtype, too few elements or not contiguous
    is refused by the binding, before the library is called."""
    S = ssamg_lib
    assert S._dptr(_FakeDeviceTensor(10), 10) == 0x1000
    assert S._dptr(_FakeDeviceTensor(12), 10) == 0x1000
    for bad in (_FakeDeviceTensor(10, "torch.float32"), _FakeDeviceTensor(9),
                _FakeDeviceTensor(10, contiguous=False)):
        with pytest.raises(ValueError):
            S._dptr(bad, 10)
    with pytest.raises(ValueError):
        S._dptr(np.zeros(10), 10)       # host memory is not a device vector


def test_num_parts_needs_a_hierarchy(ssamg_lib):
    S = ssamg_lib
    sv = S.Solver()
    assert S.lib().ssamg_num_parts(sv.h) == S.ERR_STATE
    assert S.lib().ssamg_num_parts(None) == S.ERR_STATE
    with pytest.raises(S.SsamgError):
        sv.spacings()


def test_barrier_selftest_argument_ranges(ssamg_lib):
    """Out-of-range self-test arguments are refused on the host, before any
    launch (so that no wait can be asked to poll for long)."""
    S = ssamg_lib
    L = S.lib()
    for args in ((0, 0, 10), (9, 0, 10), (2, -1, 10), (2, 1025, 10), (2, 1, 0),
                 (2, 1, (1 << 20) + 1)):
        assert L.ssamg_selftest_barrier(*args, None) == S.ERR_ARG, args


def test_grid_add_box_validation(ssamg_lib):
    """A part of several boxes: add_box after set_box only, the bounding box
    grows, couplings must leave the part (the notch is outside it)."""
    S = ssamg_lib
    L = S.lib()
    g = ctypes.c_void_p()
    assert L.ssamg_grid_create(3, 2, ctypes.byref(g)) == 0
    assert L.ssamg_grid_add_box(g, 0, S._ints([0, 4, 0]), S._ints([3, 7, 3])) == S.ERR_ARG  # no set_box yet
    assert L.ssamg_grid_set_box(g, 0, S._ints([0, 0, 0]), S._ints([7, 3, 3])) == 0
    assert L.ssamg_grid_add_box(g, 0, S._ints([0, 4, 0]), S._ints([3, 7, 3])) == 0
    assert L.ssamg_grid_add_box(g, 0, S._ints([2, 2, 2]), S._ints([1, 1, 1])) == S.ERR_ARG   # hi < lo
    assert L.ssamg_grid_set_box(g, 1, S._ints([0, 0, 0]), S._ints([3, 3, 3])) == 0
    assert L.ssamg_grid_assemble(g) == 0
    assert L.ssamg_grid_num_cells(g) == 8 * 8 * 4 + 4 ** 3     # the bounding box and the cube
    assert L.ssamg_grid_add_box(g, 1, S._ints([0, 0, 0]), S._ints([1, 1, 1])) == S.ERR_STATE
    A = ctypes.c_void_p()
    offs = [0, 0, 0, 1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1]
    assert L.ssamg_matrix_create(g, 7, S._ints(offs), ctypes.byref(A)) == 0

    def add(part, idx, d, q, nidx):
        v = np.array([-1.0])
        return L.ssamg_matrix_add_couplings(A, 1, S._ints([part]), S._ints(idx), S._ints(d),
                                            S._ints([q]), S._ints(nidx), v.ctypes.data_as(S._dp))
    assert add(0, (3, 5, 1), (1, 0, 0), 1, (0, 1, 1)) == 0         # beside the notch, leaves through +x
    assert add(0, (2, 5, 1), (1, 0, 0), 1, (0, 1, 1)) == S.ERR_ARG  # +x neighbour is in the part
    assert add(0, (5, 5, 1), (0, 0, 0), 1, (0, 1, 1)) == S.ERR_ARG  # the row is in the notch
    L.ssamg_matrix_destroy(A)
    L.ssamg_grid_destroy(g)
