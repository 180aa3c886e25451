"""Thin Python binding of the pbfmm C-ABI (include/pbfmm.h).

Argument marshalling only: every step of the computation runs in the CUDA
library libpbfmm.so built from csrc/.  Buffers may be torch tensors (device
or host) or numpy arrays (host); their raw pointers are passed through.
There is no fallback: importing this package fails if the library is absent.

Typical use (device tensors; host arrays work too and synchronise):

    import paper_2103_01048_gb300 as pb
    ctx = pb.pb_create(0, None)
    tree = pb.fmm_tree_build(ctx, xyz, 128)            # float32 [n, 3]
    pb.fmm_apply_pair(ctx, tree, 0.125, 6, out_lap, out_yuk,
                      q_lap=q, q_yuk=q, dip=d, src_n=normals)
    mesh = pb.pb_mesh_setup(ctx, verts, tris, 3, 6, 128)
    res, status = pb.pb_solve(ctx, mesh, atoms, charges, 4.0, 80.0, 0.125, 1e-6)
    dG = pb.pb_solvation_energy(ctx, res)              # kcal/mol
    pb.pb_result_destroy(res); pb.pb_mesh_destroy(mesh)
    pb.fmm_tree_destroy(tree); pb.pb_destroy(ctx)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libpbfmm.so")

if not os.path.exists(_LIBPATH):
    raise ImportError(f"libpbfmm.so not built ({_LIBPATH}); run __graft_entry__.build()")

_lib = ctypes.CDLL(_LIBPATH)

PB_OK, PB_EINVAL, PB_ENOMEM, PB_ECUDA, PB_EMESH, PB_ENOCONV, PB_ETIMEOUT = range(7)
FMM_LAPLACE, FMM_YUKAWA = 0, 1
PB_MIXED, PB_FP64 = 0, 1
_ERRNAMES = {1: "PB_EINVAL", 2: "PB_ENOMEM", 3: "PB_ECUDA", 4: "PB_EMESH", 5: "PB_ENOCONV", 6: "PB_ETIMEOUT"}

_P = ctypes.c_void_p
_I64 = ctypes.c_int64


class fmm_tree_info_t(ctypes.Structure):
    _fields_ = [("n_src", _I64), ("n_tgt", _I64), ("n_box", _I64), ("n_leaf", _I64),
                ("n_levels", ctypes.c_int32), ("same", ctypes.c_int32),
                ("n_u", _I64), ("n_v", _I64), ("n_w", _I64), ("n_x", _I64),
                ("center", ctypes.c_double * 3), ("half_width", ctypes.c_double),
                ("p2p_pairs", _I64), ("m2p_targets", _I64), ("p2l_sources", _I64), ("l2p_targets", _I64),
                ("p2m_sources", _I64), ("n_dense_box", _I64)]


def _sig(name, args, res=ctypes.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("pb_create", [ctypes.POINTER(_P), ctypes.c_int, _P])
_sig("pb_destroy", [_P])
_sig("pb_last_error", [_P], ctypes.c_char_p)
_sig("pb_sync", [_P])
_sig("pb_profile", [_P, ctypes.c_int])
_sig("pb_set_option", [_P, ctypes.c_int, ctypes.c_int])
_sig("pb_profile_read", [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)])
_sig("fmm_tree_build", [_P, _P, _I64, _P, _I64, ctypes.c_int, ctypes.POINTER(_P)])
_sig("fmm_tree_destroy", [_P])
_sig("fmm_tree_info", [_P, ctypes.POINTER(fmm_tree_info_t)])
_sig("fmm_tree_export_points", [_P, _P, _P, _P, _P])
_sig("fmm_tree_export_boxes", [_P] + [_P] * 9)
_sig("fmm_tree_export_list", [_P, ctypes.c_int, _P, _P])
_sig("fmm_apply", [_P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, _P])
_sig("fmm_apply_pair", [_P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P, _P, _P])


class pb_fmm_params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("ncrit", ctypes.c_int)]


_D = ctypes.c_double
_sig("pb_mesh_setup", [_P, _P, _I64, _P, _I64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(pb_fmm_params),
                       ctypes.POINTER(_P)])
_sig("pb_mesh_destroy", [_P])
_sig("pb_mesh_info", [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)])
_sig("pb_mesh_export_singular", [_P, _P, _D, _P, _P, _P])
_sig("pb_mesh_matvec", [_P, _P, _D, _D, _D, ctypes.c_int, ctypes.c_int, _P, _P])
_sig("pb_mesh_matvec_ex", [_P, _P, _D, _D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P])
_sig("pb_mesh_unknowns", [_P, ctypes.POINTER(_I64)])
_sig("pb_solve", [_P, _P, _P, _P, _I64, _D, _D, _D, _D, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_P)])
_sig("pb_solve_ex", [_P, _P, _P, _P, _I64, _D, _D, _D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                     ctypes.POINTER(_P)])
_sig("pb_result_destroy", [_P])
_sig("pb_result_get", [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_D), _P])
_sig("pb_solvation_energy", [_P, _P, ctypes.POINTER(_D), _P])
_sig("pb_solvation_energy_noalloc", [_P, _P, _P])
_sig("pb_energy_grad", [_P, _P, _D, ctypes.c_int, _P, _P])
_sig("pb_solve_batch", [_P, _P, ctypes.c_int, _P, _P, _P, _D, _D, _D, _D, ctypes.c_int, ctypes.c_int, _P, _P])
_sig("pb_solve_batch_ex", [_P, _P, ctypes.c_int, _P, _P, _P, _D, _D, _D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           _P, _P])
_sig("pb_tune_ncrit", [_P, _P, _I64, ctypes.c_int, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(_D)])
_sig("pb_tune", [_P, _P, _I64, ctypes.c_int, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_D)])


class PBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


def lib_path():
    return _LIBPATH


def exported_symbols():
    """Names this binding resolves in the library."""
    return ["pb_create", "pb_destroy", "pb_last_error", "pb_sync", "pb_profile", "pb_profile_read", "pb_set_option",
            "fmm_tree_build", "fmm_tree_destroy",
            "fmm_tree_info", "fmm_tree_export_points", "fmm_tree_export_boxes", "fmm_tree_export_list",
            "fmm_apply", "fmm_apply_pair", "pb_mesh_setup", "pb_mesh_destroy", "pb_mesh_info", "pb_mesh_export_singular",
            "pb_mesh_matvec", "pb_mesh_matvec_ex", "pb_mesh_unknowns", "pb_solve", "pb_solve_ex",
            "pb_result_destroy", "pb_result_get", "pb_solvation_energy",
            "pb_solvation_energy_noalloc", "pb_energy_grad", "pb_solve_batch", "pb_solve_batch_ex", "pb_tune_ncrit",
            "pb_tune"]


def ptr(x):
    """Raw pointer of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _check(rc, ctx):
    if rc != PB_OK:
        raise PBError(rc, _lib.pb_last_error(ctx).decode() if ctx else "")


def pb_create(device=0, stream=None):
    """Context on `device`; `stream` is a torch.cuda.Stream, a raw handle or None."""
    h = _P()
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(_lib.pb_create(ctypes.byref(h), int(device), s), None)
    return h


def pb_destroy(ctx):
    _check(_lib.pb_destroy(ctx), None)


def pb_sync(ctx):
    _check(_lib.pb_sync(ctx), ctx)


PHASES = ["gather", "p2m", "m2m", "p2l", "m2l", "down", "leaf", "scatter", "bem", "gmres"]
PB_PH_LAUNCHES = 100


PB_OPT_COUPLING, PB_OPT_DETERMINISTIC, PB_OPT_SINGULAR, PB_OPT_OVERLAP, PB_OPT_RESTART = 1, 2, 3, 4, 5
PB_OPT_LEAF_NT, PB_OPT_LEAF_PACKED, PB_OPT_M2L_TILE, PB_OPT_LIST_DIRECT = 6, 7, 8, 9


def pb_set_option(ctx, option, value):
    _check(_lib.pb_set_option(ctx, int(option), int(value)), ctx)


def pb_profile(ctx, enable=True):
    _check(_lib.pb_profile(ctx, 1 if enable else 0), ctx)


def pb_profile_read(ctx):
    """{phase: (ms, calls)} for every phase, plus 'launches'."""
    res = {}
    ms = ctypes.c_double()
    n = _I64()
    for i, name in enumerate(PHASES):
        _check(_lib.pb_profile_read(ctx, i, ctypes.byref(ms), ctypes.byref(n)), ctx)
        res[name] = (ms.value, n.value)
    _check(_lib.pb_profile_read(ctx, PB_PH_LAUNCHES, ctypes.byref(ms), ctypes.byref(n)), ctx)
    res["launches"] = n.value
    return res


def fmm_tree_build(ctx, src_xyz, ncrit, tgt_xyz=None):
    n = int(np.prod(src_xyz.shape)) // 3
    nt = 0 if tgt_xyz is None else int(np.prod(tgt_xyz.shape)) // 3
    h = _P()
    _check(_lib.fmm_tree_build(ctx, ptr(src_xyz), n, ptr(tgt_xyz), nt, int(ncrit), ctypes.byref(h)), ctx)
    return h


def fmm_tree_destroy(tree):
    _check(_lib.fmm_tree_destroy(tree), None)


def fmm_tree_info(tree):
    info = fmm_tree_info_t()
    _check(_lib.fmm_tree_info(tree, ctypes.byref(info)), None)
    return info


def fmm_tree_export(ctx, tree):
    """All tree arrays as numpy (for bit-exact comparison with the oracle)."""
    info = fmm_tree_info(tree)
    ns, nt, nb = info.n_src, info.n_tgt, info.n_box
    out = dict(perm_src=np.zeros(ns, np.int32), keys_src=np.zeros(ns, np.uint64),
               perm_tgt=np.zeros(nt, np.int32), keys_tgt=np.zeros(nt, np.uint64))
    _check(_lib.fmm_tree_export_points(tree, *[ptr(out[k]) for k in ("perm_src", "keys_src", "perm_tgt", "keys_tgt")]), ctx)
    names = ["level", "parent", "first_child", "nchild", "anchor", "src_begin", "src_end", "tgt_begin", "tgt_end"]
    for k in names:
        out[k] = np.zeros(nb * 3 if k == "anchor" else nb, np.int32)
    _check(_lib.fmm_tree_export_boxes(tree, *[ptr(out[k]) for k in names]), ctx)
    out["anchor"] = out["anchor"].reshape(nb, 3)
    for which, name in enumerate("UVWX"):
        off = np.zeros(nb + 1, np.int64)
        _check(_lib.fmm_tree_export_list(tree, which, ptr(off), None), ctx)
        ids = np.zeros(max(int(off[-1]), 1), np.int32)
        _check(_lib.fmm_tree_export_list(tree, which, ptr(off), ptr(ids)), ctx)
        out[name] = (off, ids[:off[-1]])
    out["info"] = info
    return out


def fmm_apply(ctx, tree, kernel, kappa, p, out, q=None, dip=None, src_n=None, tgt_n=None, out_dn=None,
              precision=PB_MIXED):
    _check(_lib.fmm_apply(ctx, tree, int(kernel), float(kappa), int(p), int(precision), ptr(q), ptr(dip),
                          ptr(src_n), ptr(tgt_n), ptr(out), ptr(out_dn)), ctx)


def fmm_apply_pair(ctx, tree, kappa, p, out_lap, out_yuk, q_lap=None, q_yuk=None, dip=None, src_n=None,
                   tgt_n=None, dn_lap=None, dn_yuk=None, precision=PB_MIXED):
    """Laplace and Yukawa potentials of the same points in one traversal."""
    _check(_lib.fmm_apply_pair(ctx, tree, float(kappa), int(p), int(precision), ptr(q_lap), ptr(q_yuk), ptr(dip),
                               ptr(src_n), ptr(tgt_n), ptr(out_lap), ptr(out_yuk), ptr(dn_lap), ptr(dn_yuk)), ctx)


PB_P0, PB_P1 = 0, 1
PB_FORM_DIRECT, PB_FORM_EXTERIOR, PB_FORM_INTERIOR = 0, 1, 2


def pb_mesh_setup(ctx, verts, tris, nquad=3, p=6, ncrit=128, basis=PB_P0):
    """verts float64 [nv,3], tris int32 [nt,3] (host numpy or device tensors)."""
    nv = int(np.prod(verts.shape)) // 3
    nt = int(np.prod(tris.shape)) // 3
    prm = pb_fmm_params(int(p), int(ncrit))
    h = _P()
    _check(_lib.pb_mesh_setup(ctx, ptr(verts), nv, ptr(tris), nt, int(basis), int(nquad), ctypes.byref(prm),
                              ctypes.byref(h)), ctx)
    return h


def pb_mesh_destroy(mesh):
    _check(_lib.pb_mesh_destroy(mesh), None)


def pb_mesh_info(mesh):
    a, b, c = _I64(), _I64(), _I64()
    _check(_lib.pb_mesh_info(mesh, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), None)
    return a.value, b.value, c.value


def pb_mesh_export_singular(ctx, mesh, kappa, p1=False):
    """(adj_off, adj_ids, S): S [nadj, 4] for a P0 mesh, [nadj, 4, 3, 3] for a P1 mesh (p1=True)."""
    nt, _, nadj = pb_mesh_info(mesh)
    off = np.zeros(nt + 1, np.int64)
    ids = np.zeros(nadj, np.int32)
    S = np.zeros((nadj, 4, 3, 3) if p1 else (nadj, 4))
    _check(_lib.pb_mesh_export_singular(ctx, mesh, float(kappa), ptr(off), ptr(ids), ptr(S)), ctx)
    return off, ids, S


def pb_mesh_matvec(ctx, mesh, x, y, eps_in, eps_out, kappa, precision=PB_MIXED, precond=False,
                   formulation=PB_FORM_DIRECT):
    _check(_lib.pb_mesh_matvec_ex(ctx, mesh, float(eps_in), float(eps_out), float(kappa), int(precision),
                                  1 if precond else 0, int(formulation), ptr(x), ptr(y)), ctx)


def pb_mesh_unknowns(mesh):
    """Unknowns per block: triangles (P0) or vertices (P1)."""
    n = _I64()
    _check(_lib.pb_mesh_unknowns(mesh, ctypes.byref(n)), None)
    return n.value


def pb_solve(ctx, mesh, atoms, charges, eps_in, eps_out, kappa, tol, max_iter=500, precision=PB_MIXED,
             formulation=PB_FORM_DIRECT):
    """Returns (result handle, status); status PB_OK or PB_ENOCONV (handle valid in both)."""
    atoms = np.ascontiguousarray(atoms, dtype=np.float64) if isinstance(atoms, np.ndarray) else atoms
    charges = np.ascontiguousarray(charges, dtype=np.float64) if isinstance(charges, np.ndarray) else charges
    na = int(np.prod(charges.shape))
    h = _P()
    rc = _lib.pb_solve_ex(ctx, mesh, ptr(atoms), ptr(charges), na, float(eps_in), float(eps_out), float(kappa),
                          float(tol), int(max_iter), int(precision), int(formulation), ctypes.byref(h))
    if rc not in (PB_OK, PB_ENOCONV) or not h:
        _check(rc, ctx)
    return h, rc


def pb_result_get(res, n=None):
    """(iterations, residual, x); x [2 n] when n (pb_mesh_unknowns) is given."""
    it = ctypes.c_int()
    rr = _D()
    x = None
    if n is not None:
        x = np.zeros(2 * n)
    _check(_lib.pb_result_get(res, ctypes.byref(it), ctypes.byref(rr), ptr(x)), None)
    return it.value, rr.value, x


def pb_result_destroy(res):
    _check(_lib.pb_result_destroy(res), None)


def pb_solvation_energy(ctx, res, na=None):
    e = _D()
    phir = np.zeros(na) if na else None
    _check(_lib.pb_solvation_energy(ctx, res, ctypes.byref(e), ptr(phir)), ctx)
    return (e.value, phir) if na else e.value


def pb_solvation_energy_noalloc(ctx, res, dG_device, device=None):
    """Energy into a caller-owned device double without any device
    allocation; asynchronous on the context stream.  dG_device must be a
    CUDA torch tensor of dtype float64 with at least one element on the
    context's device (`device`, default the current CUDA device)."""
    if not (hasattr(dG_device, "is_cuda") and dG_device.is_cuda):
        raise ValueError("dG_device must be a CUDA tensor")
    import torch
    if dG_device.dtype != torch.float64 or dG_device.numel() < 1:
        raise ValueError("dG_device must be float64 with at least one element")
    want = torch.cuda.current_device() if device is None else int(device)
    if dG_device.device.index != want:
        raise ValueError(f"dG_device is on cuda:{dG_device.device.index}, the context on cuda:{want}")
    _check(_lib.pb_solvation_energy_noalloc(ctx, res, ptr(dG_device)), ctx)


def pb_energy_grad(ctx, res, na, tol=1e-8, max_iter=500):
    """(dE/dq [na], dE/dx [na,3]) in kcal/mol/e and kcal/mol/A; raises on failure."""
    gq = np.zeros(na)
    gx = np.zeros((na, 3))
    rc = _lib.pb_energy_grad(ctx, res, float(tol), int(max_iter), ptr(gq), ptr(gx))
    if rc not in (PB_OK, PB_ENOCONV):
        _check(rc, ctx)
    return gq, gx, rc


def pb_solve_batch(ctx, meshes, atoms_list, charges_list, eps_in, eps_out, kappa, tol, max_iter=500,
                   precision=PB_MIXED, formulation=None):
    """Solve len(meshes) systems together; returns (results, statuses, rc).
    formulation (PB_FORM_*; None: the direct formulation through
    pb_solve_batch) selects pb_solve_batch_ex."""
    ns = len(meshes)
    A = [np.ascontiguousarray(a, dtype=np.float64) for a in atoms_list]
    Q = [np.ascontiguousarray(q, dtype=np.float64) for q in charges_list]
    mesh_arr = (_P * ns)(*[m.value if isinstance(m, _P) else m for m in meshes])
    a_arr = (_P * ns)(*[a.ctypes.data for a in A])
    q_arr = (_P * ns)(*[q.ctypes.data for q in Q])
    na = np.array([len(q) for q in Q], dtype=np.int64)
    out = (_P * ns)()
    st = np.zeros(ns, dtype=np.int32)
    if formulation is None:
        rc = _lib.pb_solve_batch(ctx, mesh_arr, ns, a_arr, q_arr, ptr(na), float(eps_in), float(eps_out),
                                 float(kappa), float(tol), int(max_iter), int(precision), out, ptr(st))
    else:
        rc = _lib.pb_solve_batch_ex(ctx, mesh_arr, ns, a_arr, q_arr, ptr(na), float(eps_in), float(eps_out),
                                    float(kappa), float(tol), int(max_iter), int(precision), int(formulation), out,
                                    ptr(st))
    if rc not in (PB_OK, PB_ENOCONV):
        _check(rc, ctx)
    return [_P(out[i]) for i in range(ns)], st, rc


def pb_tune_ncrit(ctx, xyz, p, candidates):
    """(best ncrit, its ms) for one Laplace + one Yukawa SL+DL apply."""
    cand = np.ascontiguousarray(candidates, dtype=np.int32)
    best = ctypes.c_int()
    ms = _D()
    n = int(np.prod(xyz.shape)) // 3
    _check(_lib.pb_tune_ncrit(ctx, ptr(xyz), n, int(p), ptr(cand), len(cand), ctypes.byref(best), ctypes.byref(ms)),
           ctx)
    return best.value, ms.value


def pb_tune(ctx, xyz, p, candidates):
    """(best ncrit, leaf targets per thread, M2L tile option, its ms) for the
    paired Laplace + Yukawa SL+DL apply; the context keeps the best tile options."""
    cand = np.ascontiguousarray(candidates, dtype=np.int32)
    best, nt, tile = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms = _D()
    n = int(np.prod(xyz.shape)) // 3
    _check(_lib.pb_tune(ctx, ptr(xyz), n, int(p), ptr(cand), len(cand), ctypes.byref(best), ctypes.byref(nt),
                        ctypes.byref(tile), ctypes.byref(ms)), ctx)
    return best.value, nt.value, tile.value, ms.value


# test hooks (include/pbfmm_testing.h; not part of the solver's interface)
_lib.pbfmm_selftest_m2l_tc.argtypes = [ctypes.c_int, ctypes.c_int, _P, _P, _P]
_lib.pbfmm_selftest_m2l_tc.restype = ctypes.c_int
_lib.pbfmm_test_alloc_count.argtypes = []
_lib.pbfmm_test_alloc_count.restype = _I64
_lib.pbfmm_test_fail_alloc.argtypes = [_I64]
_lib.pbfmm_test_fail_alloc.restype = None
_lib.pbfmm_test_wait_limit.argtypes = [_I64]
_lib.pbfmm_test_wait_limit.restype = None
_lib.pbfmm_test_radix_sort.argtypes = [_P, _P, _I64, ctypes.c_int, _P, _P]
_lib.pbfmm_test_radix_sort.restype = ctypes.c_int
_lib.pbfmm_test_sym_eig.argtypes = [ctypes.c_int, _P, _P, _P]
_lib.pbfmm_test_sym_eig.restype = ctypes.c_int
_lib.pbfmm_test_tc_pair_info.argtypes = [_P]
_lib.pbfmm_test_tc_pair_info.restype = ctypes.c_int
_lib.pbfmm_test_tc_pair.argtypes = [ctypes.c_int]
_lib.pbfmm_test_tc_pair.restype = ctypes.c_int
_lib.pbfmm_test_pool_used.argtypes = [ctypes.c_int]
_lib.pbfmm_test_pool_used.restype = _I64


def _test_radix_sort(keys, vals, bits):
    """(sorted keys, values) by the library's stable radix sort (uint64 keys, int32 values)."""
    k = np.ascontiguousarray(keys, np.uint64)
    v = np.ascontiguousarray(vals, np.int32)
    ko = np.zeros_like(k)
    vo = np.zeros_like(v)
    rc = _lib.pbfmm_test_radix_sort(ptr(k), ptr(v), len(k), int(bits), ptr(ko), ptr(vo))
    if rc != PB_OK:
        raise PBError(rc, "radix sort failed")
    return ko, vo


def _test_pool_used(device=0):
    """Bytes in use (not cached) in the device's default stream-ordered pool."""
    return int(_lib.pbfmm_test_pool_used(int(device)))


def _test_sym_eig(A):
    """(w, V) of a symmetric matrix from the library's host eigensolver."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n))
    rc = _lib.pbfmm_test_sym_eig(n, ptr(A), ptr(w), ptr(V))
    if rc != PB_OK:
        raise PBError(rc, "sym_eig")
    return w, V


def _test_tc_pair_info():
    """Launch properties of the CTA-pair kernel (npad 128): registers, max
    threads per block, static and dynamic shared bytes, resident clusters."""
    out = np.zeros(5, dtype=np.int32)
    rc = _lib.pbfmm_test_tc_pair_info(ptr(out))
    if rc != PB_OK:
        raise PBError(rc, "tc pair info")
    return dict(zip(("regs", "max_threads", "static_smem", "dyn_smem", "max_active_clusters"), out.tolist()))


def _test_tc_pair(mode):
    """Select the tensor-core box-operator kernel (1: CTA pairs where
    available, 0: one CTA per operator part); returns the previous mode."""
    return int(_lib.pbfmm_test_tc_pair(int(mode)))


def _test_alloc_count():
    """Device allocations the library has made so far."""
    return int(_lib.pbfmm_test_alloc_count())


def _test_fail_alloc(nth):
    """Make the nth device allocation from now fail with PB_ENOMEM (0: off)."""
    _lib.pbfmm_test_fail_alloc(int(nth))


def _test_wait_limit(cycles):
    """Cycle limit of the tensor-core kernel's bounded waits (<= 0: default)."""
    _lib.pbfmm_test_wait_limit(int(cycles))


def _selftest_m2l_tc(Q, Op):
    """D = Q Op^T through the tcgen05 M2L kernel (float32 host arrays)."""
    Q = np.ascontiguousarray(Q, np.float32)
    Op = np.ascontiguousarray(Op, np.float32)
    D = np.zeros_like(Q)
    rc = _lib.pbfmm_selftest_m2l_tc(Q.shape[0], Q.shape[1], ptr(Q), ptr(Op), ptr(D))
    if rc != PB_OK:
        raise PBError(rc, "tensor-core M2L self-test failed")
    return D


# arithmetic-pipe microbenchmarks (include/pbfmm_peaks.h)
_lib.pbfmm_measure_peaks.argtypes = [ctypes.c_int, _P]
_lib.pbfmm_measure_peaks.restype = ctypes.c_int
PEAK_KEYS = ("fp32_fma_tflops", "mufu_rsqrt_tops", "mufu_ex2_tops", "fp64_fma_tflops", "tf32_tc_tflops",
             "bf16_tc_tflops", "fp32x2_fma_tflops")


def measure_peaks(device=0):
    """Measured rates of the FP32 FMA pipe (scalar and packed f32x2), the MUFU
    rsqrt and ex2 units, FP64 FMA and the tcgen05 TF32 / BF16 tensor cores on
    `device` (dict, units in the key names: TFLOP/s or 10^12 results/s)."""
    out = np.zeros(7)
    rc = _lib.pbfmm_measure_peaks(int(device), ptr(out))
    if rc != PB_OK:
        raise PBError(rc, "peak microbenchmarks failed")
    return dict(zip(PEAK_KEYS, (float(v) for v in out)))

