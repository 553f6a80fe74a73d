"""TEST INFRASTRUCTURE: ctypes wrapper around the C oracle (rbffd_oracle.c).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg import
this module.  It is the plain sequential FP64 restatement of the overlapped RBF-FD
construction (§2, §4.1, §4.2.1) that the CUDA library is checked against; the CUDA library
never loads it.  The shared object is compiled on first use with gcc -ffp-contract=off.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rbffd_oracle.c")
# RBFFD_ORACLE_TEST_LIB: a prebuilt copy of the oracle with a planted mistake, used by the test
# that checks every such mistake fails a pin (never set otherwise)
_TEST_LIB = os.environ.get("RBFFD_ORACLE_TEST_LIB")
LIB = _TEST_LIB or os.path.join(HERE, "_build", "liboracle.so")

OK, EINVAL, EDUPLICATE, ENOMEM, ESINGULAR = 0, -1, -2, -3, -4
OP_LAPLACIAN, OP_IDENTITY, OP_NORMAL = 0, 1, 2
STAB_SEQ, STAB_OFF, STAB_FALLBACK = 0, 1, 2
LREF_CENTER, LREF_CENTROID = 0, 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain C, FP64, no FMA contraction)."""
    if _TEST_LIB:
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    stale = (not os.path.exists(LIB)) or os.path.getmtime(LIB) < max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "rbffd_oracle.h")))
    if force or stale:
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Stats(C.Structure):
    _fields_ = [("n_centers", C.c_int64), ("n_fallback", C.c_int64),
                ("n_decisions", C.c_int64), ("n_rejected", C.c_int64),
                ("n_near_tie", C.c_int64), ("sum_q", C.c_int64), ("sum_cols", C.c_int64),
                ("min_abs_margin", C.c_double), ("n_boundary", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            P = C.c_void_p
            L.ora_degree_for_n.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int)]
            L.ora_poly_terms.argtypes = [C.c_int, C.c_int, P]
            L.ora_knn.argtypes = [P, C.c_int64, C.c_int, C.c_int, P, P]
            L.ora_ball_len.argtypes = [P, C.c_int64, C.c_int, C.c_double, P]
            L.ora_local_weights.argtypes = [P, C.c_int, P, C.c_int, C.c_int, C.c_int, C.c_int,
                                            P, C.c_int, P, P]
            L.ora_assemble.argtypes = [P, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int,
                                       C.c_double, C.c_int, P, P, P, P, P, P, P, P,
                                       C.POINTER(Stats)]
            L.ora_local_weights_dn.argtypes = [P, C.c_int, P, C.c_int, C.c_int, C.c_int, C.c_int,
                                               P, P, C.c_int, P, P]
            L.ora_assemble_bc.argtypes = [P, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int,
                                          C.c_double, C.c_int, C.c_int, P, P, P, P, P, P, P, P,
                                          P, P, C.POINTER(Stats)]
            L.ora_assemble_mixed.argtypes = [P, C.c_int64, C.c_int, P, P, P, C.c_int,
                                             C.c_double, C.c_int, C.c_int, P, P, P, P, P, P, P,
                                             P, C.POINTER(Stats)]
            _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: oracle error {code}")
        self.code = code


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _check(rc, what):
    if rc != OK:
        raise OracleError(rc, what)


def degree_for_n(n: int, d: int):
    """(s, M) from the degree rule of §2."""
    M = C.c_int(0)
    s = lib().ora_degree_for_n(n, d, C.byref(M))
    _check(0 if s >= 0 else s, "degree_for_n")
    return s, M.value


def poly_terms(d: int, ell: int) -> np.ndarray:
    M = lib().ora_poly_terms(d, ell, None)
    e = np.zeros((M, d), dtype=np.int32)
    lib().ora_poly_terms(d, ell, _ptr(e))
    return e


def knn(X: np.ndarray, n: int):
    """Brute-force kNN table (nbr [N][n] int32, d2 [N][n] float64)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    N, d = X.shape
    nbr = np.zeros((N, n), dtype=np.int32)
    d2 = np.zeros((N, n), dtype=np.float64)
    _check(lib().ora_knn(_ptr(X), N, d, n, _ptr(nbr), _ptr(d2)), "knn")
    return nbr, d2


def ball_len(d2: np.ndarray, delta: float) -> np.ndarray:
    d2 = np.ascontiguousarray(d2, dtype=np.float64)
    N, n = d2.shape
    out = np.zeros(N, dtype=np.int32)
    _check(lib().ora_ball_len(_ptr(d2), N, n, float(delta), _ptr(out)), "ball_len")
    return out


def local_weights(X, idx, ell, m, Y, op=OP_LAPLACIAN):
    """Weights W [n][q] of stencil X[idx] (idx[0] = center) for operator op at points Y [q][d],
    and the scaled local Lebesgue values lam [q]."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    Y = np.ascontiguousarray(np.atleast_2d(Y), dtype=np.float64)
    d = X.shape[1]
    n = idx.size
    q = Y.shape[0]
    W = np.zeros((n, q), dtype=np.float64)
    lam = np.zeros(q, dtype=np.float64)
    _check(lib().ora_local_weights(_ptr(X), d, _ptr(idx), n, ell, m, op, _ptr(Y), q,
                                   _ptr(W), _ptr(lam)), "local_weights")
    return W, lam


def normal_weights(X, idx, ell, m, nrm):
    """Weights W [n] of stencil X[idx] for the derivative along the unit vector nrm at the
    center X[idx[0]] (the Neumann operator), and the scaled local Lebesgue value."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    d = X.shape[1]
    n = idx.size
    Y = np.ascontiguousarray(X[idx[0]][None, :])
    Nr = np.ascontiguousarray(np.asarray(nrm, dtype=np.float64).reshape(1, d))
    W = np.zeros(n, dtype=np.float64)
    lam = np.zeros(1, dtype=np.float64)
    _check(lib().ora_local_weights_dn(_ptr(X), d, _ptr(idx), n, ell, m, OP_NORMAL, _ptr(Y),
                                      _ptr(Nr), 1, _ptr(W), _ptr(lam)), "local_weights_dn")
    return W, lam[0]


def assemble(X, n, ell, m, delta, mode=STAB_SEQ, nbr=None, d2=None, bc=None, normals=None,
             lref=LREF_CENTER):
    """The whole sequential construction of L.  Returns a dict with CSR arrays (row_ptr, col,
    val), owner, is_center, lam_row, stats and the kNN table used.  bc (uint8 [N]: 0
    interior, 1 Dirichlet, 2 Neumann) and normals ([N][d]) add the boundary rows of §5.
    lref picks the reference point of the Lebesgue test (§4.2.1): the stencil's center, or
    with LREF_CENTROID the stencil node nearest the stencil's centroid."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    N, d = X.shape
    if nbr is None or d2 is None:
        nbr, d2 = knn(X, n)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    col = np.zeros(N * n, dtype=np.int32)
    val = np.zeros(N * n, dtype=np.float64)
    owner = np.zeros(N, dtype=np.int32)
    is_center = np.zeros(N, dtype=np.uint8)
    lam_row = np.zeros(N, dtype=np.float64)
    st = Stats()
    bcv = None if bc is None else np.ascontiguousarray(bc, dtype=np.uint8)
    nrv = None if normals is None else np.ascontiguousarray(normals, dtype=np.float64)
    _check(lib().ora_assemble_bc(_ptr(X), N, d, n, ell, m, float(delta), mode, lref, _ptr(bcv),
                                 _ptr(nrv), _ptr(np.ascontiguousarray(nbr, dtype=np.int32)),
                                 _ptr(np.ascontiguousarray(d2, dtype=np.float64)),
                                 _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(owner),
                                 _ptr(is_center), _ptr(lam_row), C.byref(st)), "assemble")
    return dict(row_ptr=row_ptr, col=col, val=val, owner=owner, is_center=is_center,
                lam_row=lam_row, stats=st.as_dict(), nbr=nbr, d2=d2)


def assemble_mixed(X, n_node, ell_node, m_node, delta, mode=STAB_SEQ, nbr=None, d2=None,
                   lref=LREF_CENTER):
    """The traversal with per-node stencil size, degree and PHS exponent.  Returns the same
    dict as assemble(); CSR rows have the length of the stencil that produced them."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    N, d = X.shape
    n_node = np.ascontiguousarray(n_node, dtype=np.int32)
    ell_node = np.ascontiguousarray(ell_node, dtype=np.int32)
    m_node = np.ascontiguousarray(m_node, dtype=np.int32)
    n_max = int(n_node.max())
    if nbr is None or d2 is None:
        nbr, d2 = knn(X, n_max)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    col = np.zeros(N * n_max, dtype=np.int32)
    val = np.zeros(N * n_max, dtype=np.float64)
    owner = np.zeros(N, dtype=np.int32)
    is_center = np.zeros(N, dtype=np.uint8)
    lam_row = np.zeros(N, dtype=np.float64)
    st = Stats()
    _check(lib().ora_assemble_mixed(_ptr(X), N, d, _ptr(n_node), _ptr(ell_node), _ptr(m_node),
                                    n_max, float(delta), mode, lref,
                                    _ptr(np.ascontiguousarray(nbr, dtype=np.int32)),
                                    _ptr(np.ascontiguousarray(d2, dtype=np.float64)),
                                    _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(owner),
                                    _ptr(is_center), _ptr(lam_row), C.byref(st)),
           "assemble_mixed")
    nnz = int(row_ptr[-1])
    return dict(row_ptr=row_ptr, col=col[:nnz], val=val[:nnz], owner=owner,
                is_center=is_center, lam_row=lam_row, stats=st.as_dict(), nbr=nbr, d2=d2)


def csr_matvec(row_ptr, col, val, u):
    """y = L u for a CSR matrix (plain numpy; used to check the library's apply)."""
    y = np.zeros(row_ptr.size - 1)
    contrib = val * u[col]
    np.add.at(y, np.repeat(np.arange(row_ptr.size - 1), np.diff(row_ptr)), contrib)
    return y
