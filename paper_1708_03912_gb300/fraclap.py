"""Python binding of libfraclap (include/fraclap.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; PyTorch supplies
device memory and the current stream.  The functions carry the C names
(fl_create, fl_assemble, ...); `Mesh` is a small convenience wrapper around a
handle.  There is no CPU path: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfraclap.so")

FL_OK, FL_EINVAL, FL_ENOMEM, FL_ECUDA, FL_ENOTSPD, FL_ENOTCONV, FL_ETIMEOUT, FL_ENOTIMPL = range(8)
FL_DOF_INTERIOR, FL_DOF_PAPER = 0, 1
FL_FP64, FL_MIXED = 0, 1
FL_F64, FL_F32, FL_BF16, FL_F32X2 = 0, 1, 2, 3
_CODES = {0: "FL_OK", 1: "FL_EINVAL", 2: "FL_ENOMEM", 3: "FL_ECUDA", 4: "FL_ENOTSPD", 5: "FL_ENOTCONV",
          6: "FL_ETIMEOUT", 7: "FL_ENOTIMPL"}

EXPORTS = ["fl_default_options", "fl_create", "fl_create_sector", "fl_destroy", "fl_last_error", "fl_num_dofs", "fl_dof_vertices",
           "fl_assemble", "fl_tune_assemble", "fl_set_far_variant", "fl_assemble_nearfield_csr", "fl_load_vector", "fl_matvec", "fl_convert", "fl_default_solve_opts", "fl_solve",
           "fl_heat_matrix", "fl_mass_apply", "fl_strong_form", "fl_br_indicators", "fl_mark_max", "fl_refine",
           "fl_cluster_plan", "fl_near_region_plan", "fl_near_region_tiles", "fl_strong_form_cluster_plan", "fl_hmatrix_create", "fl_hmatrix_set_near",
           "fl_hmatrix_matvec", "fl_hmatrix_solve", "fl_hmatrix_info", "fl_hmatrix_assemble_near", "fl_hmatrix_near_info", "fl_hmatrix_get_near",
           "fl_hmatrix_strong_form", "fl_hmatrix_br_indicators", "fl_hmatrix_solve_shifted", "fl_hmatrix_last_error", "fl_hmatrix_destroy", "fl_get_stats", "fl_set_profiling", "fl_stage_ms", "fl_launch_count", "fl_pool_trim", "fl_pool_stats",
           "fl_matvec_f32_static",
           "fl_split_bf16_bytes", "fl_split_bf16", "fl_matmul_bf16", "fl_default_batch_opts", "fl_batch_solve",
           "fl_tune_batch", "fl_tune_matvec", "fl_tune_record", "fl_tune_lookup", "fl_tune_clear", "fl_tune_count", "fl_tune_save",
           "fl_tune_load", "fl_prolongation", "fl_mg_create", "fl_mg_add_level", "fl_mg_setup", "fl_mg_level", "fl_mg_level_copy",
           "fl_mg_omega", "fl_mg_vcycle", "fl_mg_solve", "fl_mg_last_error", "fl_mg_destroy",
           "fl_patches", "fl_lp_create", "fl_lp_num_params", "fl_lp_num_features", "fl_lp_num_samples",
           "fl_lp_get_params", "fl_lp_set_params", "fl_lp_stencil", "fl_lp_bind", "fl_lp_features", "fl_lp_apply", "fl_lp_loss_grad",
           "fl_lp_add_pairs", "fl_lp_collect", "fl_lp_collect_noise", "fl_lp_train", "fl_lp_last_error", "fl_lp_destroy", "fl_fcg_solve"]
FL_STATIC_MAX_N = 65536
FL_BATCH_MAXPROB = 8
FL_RESID_F64, FL_RESID_DF = 0, 1
STAGES = ["prep", "far", "near", "touch", "bnd", "element", "compose"]


class FlError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class fl_options(ctypes.Structure):
    _fields_ = [("k_far", ctypes.c_int), ("k_near", ctypes.c_int), ("k_touch", ctypes.c_int),
                ("k_bnd", ctypes.c_int), ("regional", ctypes.c_int), ("k_vertex", ctypes.c_int),
                ("far_f64_pipe", ctypes.c_int)]


class fl_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("inner_dtype", ctypes.c_int),
                ("A_lo_dev", ctypes.c_void_p), ("ld_lo", ctypes.c_int64), ("inner_tol", ctypes.c_double),
                ("inner_maxit", ctypes.c_int), ("barrier_timeout_us", ctypes.c_int)]


class fl_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "n_cells", "n_vertices", "n_facets", "n_dofs", "n_tiles", "n_touch_pairs", "n_near_pairs", "n_far_pairs",
        "n_cells_with_dof", "nnz_nearfield", "h2d_bytes", "workspace_bytes")]


class fl_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("status", ctypes.c_int)]


class fl_fcg_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("fallback_at", ctypes.c_int), ("final_preconditioner", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("status", ctypes.c_int)]


class fl_batch_problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("A_dev", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("S_dev", ctypes.c_void_p), ("nslices", ctypes.c_int),
                ("dscale_dev", ctypes.c_void_p), ("nrhs", ctypes.c_int), ("B_dev", ctypes.c_void_p),
                ("ldb", ctypes.c_int64), ("U_dev", ctypes.c_void_p), ("ldu", ctypes.c_int64)]


class fl_batch_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_outer", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("inner_maxit", ctypes.c_int), ("ctas", ctypes.c_int), ("stages", ctypes.c_int),
                ("barrier_timeout_us", ctypes.c_int), ("residual", ctypes.c_int)]


class fl_batch_info(ctypes.Structure):
    _fields_ = [("outer_iterations", ctypes.c_int), ("inner_iterations", ctypes.c_int), ("status", ctypes.c_int),
                ("ctas", ctypes.c_int), ("stages", ctypes.c_int)]


_lib = None


def lib():
    """Load libfraclap.so (built in-tree by __graft_entry__.build()); raise if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dbl, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int
    L.fl_default_options.argtypes = [ctypes.POINTER(fl_options)]
    L.fl_default_options.restype = None
    L.fl_create.argtypes = [ctypes.POINTER(vp), ci, i64, vp, i64, vp, ci, ctypes.POINTER(fl_options)]
    L.fl_create.restype = ci
    L.fl_destroy.argtypes = [vp]
    L.fl_destroy.restype = None
    L.fl_last_error.argtypes = [vp]
    L.fl_last_error.restype = ctypes.c_char_p
    L.fl_num_dofs.argtypes = [vp, dbl, ctypes.POINTER(i64)]
    L.fl_num_dofs.restype = ci
    L.fl_dof_vertices.argtypes = [vp, dbl, vp]
    L.fl_dof_vertices.restype = ci
    L.fl_assemble.argtypes = [vp, dbl, ci, vp, i64, vp]
    L.fl_assemble.restype = ci
    L.fl_tune_assemble.argtypes = [vp, dbl, vp, i64, ci, ctypes.POINTER(ci), ctypes.POINTER(dbl), vp]
    L.fl_tune_assemble.restype = ci
    L.fl_set_far_variant.argtypes = [vp, ci]
    L.fl_set_far_variant.restype = ci
    L.fl_assemble_nearfield_csr.argtypes = [vp, dbl, ci, ctypes.POINTER(i64), vp, vp, vp, vp]
    L.fl_assemble_nearfield_csr.restype = ci
    L.fl_load_vector.argtypes = [vp, dbl, vp, ci, vp, i64, vp]
    L.fl_load_vector.restype = ci
    L.fl_matvec.argtypes = [ci, vp, i64, i64, ci, vp, i64, vp, i64, vp]
    L.fl_matvec.restype = ci
    L.fl_convert.argtypes = [vp, i64, i64, ci, vp, i64, vp]
    L.fl_convert.restype = ci
    L.fl_heat_matrix.argtypes = [vp, dbl, dbl, vp, i64, vp, i64, vp]
    L.fl_heat_matrix.restype = ci
    L.fl_mass_apply.argtypes = [vp, dbl, ci, dbl, vp, i64, dbl, vp, i64, vp, i64, vp]
    L.fl_mass_apply.restype = ci
    L.fl_create_sector.argtypes = [ctypes.POINTER(ctypes.c_void_p), i64, vp, i64, vp, ci, vp]
    L.fl_create_sector.restype = ci
    L.fl_strong_form.argtypes = [vp, dbl, vp, ci, ci, ci, vp, vp]
    L.fl_strong_form.restype = ci
    L.fl_br_indicators.argtypes = [vp, dbl, vp, vp, ci, ci, ci, vp, vp, vp]
    L.fl_br_indicators.restype = ci
    L.fl_mark_max.argtypes = [vp, dbl, vp, dbl, vp, vp, vp]
    L.fl_mark_max.restype = ci
    L.fl_refine.argtypes = [ci, i64, vp, i64, vp, vp, i64, i64, vp, vp, ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(ctypes.c_int64)]
    L.fl_refine.restype = ci
    L.fl_cluster_plan.argtypes = [vp, dbl, dbl, ci, ctypes.POINTER(i64), vp, vp, vp, vp]
    L.fl_cluster_plan.restype = ci
    L.fl_near_region_plan.argtypes = [vp, dbl, dbl, ci, ctypes.POINTER(i64), vp, vp, vp, vp, vp, vp]
    L.fl_near_region_plan.restype = ci
    L.fl_near_region_tiles.argtypes = [vp, dbl, dbl, ci, ctypes.POINTER(i64), vp, vp]
    L.fl_near_region_tiles.restype = ci
    L.fl_strong_form_cluster_plan.argtypes = [vp, dbl, dbl, ci, ci, ctypes.POINTER(i64), vp, vp, vp, vp, vp]
    L.fl_strong_form_cluster_plan.restype = ci
    L.fl_hmatrix_create.argtypes = [vp, dbl, ci, dbl, ci, ctypes.POINTER(vp), vp]
    L.fl_hmatrix_create.restype = ci
    L.fl_hmatrix_set_near.argtypes = [vp, vp, i64, vp]
    L.fl_hmatrix_set_near.restype = ci
    L.fl_hmatrix_matvec.argtypes = [vp, vp, vp, vp]
    L.fl_hmatrix_matvec.restype = ci
    L.fl_hmatrix_solve.argtypes = [vp, vp, vp, ctypes.POINTER(fl_solve_opts), ctypes.POINTER(fl_solve_info), vp]
    L.fl_hmatrix_solve.restype = ci
    L.fl_hmatrix_info.argtypes = [vp, ctypes.POINTER(i64)]
    L.fl_hmatrix_info.restype = ci
    L.fl_hmatrix_assemble_near.argtypes = [vp, ci, vp]
    L.fl_hmatrix_assemble_near.restype = ci
    L.fl_hmatrix_near_info.argtypes = [vp, ctypes.POINTER(i64)]
    L.fl_hmatrix_near_info.restype = ci
    L.fl_hmatrix_get_near.argtypes = [vp, ctypes.POINTER(i64), vp, vp, vp, vp]
    L.fl_hmatrix_get_near.restype = ci
    L.fl_hmatrix_solve_shifted.argtypes = [vp, dbl, dbl, vp, vp, ctypes.POINTER(fl_solve_opts),
                                           ctypes.POINTER(fl_solve_info), vp]
    L.fl_hmatrix_solve_shifted.restype = ci
    L.fl_hmatrix_strong_form.argtypes = [vp, vp, ci, ci, ci, vp, vp]
    L.fl_hmatrix_strong_form.restype = ci
    L.fl_hmatrix_br_indicators.argtypes = [vp, vp, vp, ci, ci, ci, vp, vp, vp]
    L.fl_hmatrix_br_indicators.restype = ci
    L.fl_hmatrix_last_error.argtypes = [vp]
    L.fl_hmatrix_last_error.restype = ctypes.c_char_p
    L.fl_hmatrix_destroy.argtypes = [vp]
    L.fl_hmatrix_destroy.restype = None
    L.fl_default_solve_opts.argtypes = [ctypes.POINTER(fl_solve_opts)]
    L.fl_default_solve_opts.restype = None
    L.fl_solve.argtypes = [vp, i64, vp, i64, vp, vp, ctypes.POINTER(fl_solve_opts), ctypes.POINTER(fl_solve_info), vp]
    L.fl_solve.restype = ci
    L.fl_get_stats.argtypes = [vp, dbl, ctypes.POINTER(fl_stats)]
    L.fl_get_stats.restype = ci
    L.fl_set_profiling.argtypes = [vp, ci]
    L.fl_set_profiling.restype = ci
    L.fl_stage_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.fl_stage_ms.restype = ci
    L.fl_launch_count.argtypes = []
    L.fl_launch_count.restype = ctypes.c_uint64
    L.fl_pool_trim.argtypes = []
    L.fl_pool_trim.restype = i64
    L.fl_pool_stats.argtypes = [ctypes.POINTER(i64)] * 4
    L.fl_pool_stats.restype = None
    L.fl_matvec_f32_static.argtypes = [vp, i64, i64, vp, vp, vp]
    L.fl_matvec_f32_static.restype = ci
    L.fl_split_bf16_bytes.argtypes = [i64, ci]
    L.fl_split_bf16_bytes.restype = i64
    L.fl_split_bf16.argtypes = [vp, i64, i64, ci, vp, vp, vp]
    L.fl_split_bf16.restype = ci
    L.fl_matmul_bf16.argtypes = [vp, i64, ci, ci, vp, i64, vp, i64, vp]
    L.fl_matmul_bf16.restype = ci
    L.fl_default_batch_opts.argtypes = [ctypes.POINTER(fl_batch_opts)]
    L.fl_default_batch_opts.restype = None
    L.fl_batch_solve.argtypes = [vp, ci, ctypes.POINTER(fl_batch_problem), ctypes.POINTER(fl_batch_opts),
                                 ctypes.POINTER(fl_batch_info), vp, vp, vp]
    L.fl_batch_solve.restype = ci
    L.fl_tune_batch.argtypes = [vp, ci, ctypes.POINTER(fl_batch_problem), ci, ctypes.POINTER(fl_batch_opts),
                                ctypes.POINTER(dbl)]
    L.fl_tune_batch.restype = ci
    L.fl_tune_matvec.argtypes = [ci, vp, i64, i64, vp, vp, ci, ctypes.POINTER(ci), ctypes.POINTER(dbl), vp]
    L.fl_tune_matvec.restype = ci
    L.fl_tune_record.argtypes = [ctypes.c_char_p, i64, ci, ci, ci, ci, dbl]
    L.fl_tune_record.restype = ci
    L.fl_tune_lookup.argtypes = [ctypes.c_char_p, i64, ci, ci, ctypes.POINTER(ci), ctypes.POINTER(ci)]
    L.fl_tune_lookup.restype = ci
    L.fl_tune_clear.argtypes = []
    L.fl_tune_clear.restype = None
    L.fl_tune_count.argtypes = []
    L.fl_tune_count.restype = ci
    L.fl_tune_save.argtypes = [ctypes.c_char_p]
    L.fl_tune_save.restype = ci
    L.fl_tune_load.argtypes = [ctypes.c_char_p]
    L.fl_tune_load.restype = ci
    L.fl_prolongation.argtypes = [vp, vp, dbl, ctypes.POINTER(i64), vp, vp, vp]
    L.fl_prolongation.restype = ci
    L.fl_mg_create.argtypes = [ctypes.POINTER(vp), vp, i64, i64]
    L.fl_mg_create.restype = ci
    L.fl_mg_add_level.argtypes = [vp, i64, i64, vp, vp, vp, vp]
    L.fl_mg_add_level.restype = ci
    L.fl_mg_setup.argtypes = [vp, ci, vp]
    L.fl_mg_setup.restype = ci
    L.fl_mg_level.argtypes = [vp, ci, ctypes.POINTER(i64), ctypes.POINTER(vp), ctypes.POINTER(i64)]
    L.fl_mg_level.restype = ci
    L.fl_mg_level_copy.argtypes = [vp, ci, vp, i64, vp]
    L.fl_mg_level_copy.restype = ci
    L.fl_mg_omega.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_float)]
    L.fl_mg_omega.restype = ci
    L.fl_mg_vcycle.argtypes = [vp, vp, vp, vp]
    L.fl_mg_vcycle.restype = ci
    L.fl_mg_solve.argtypes = [vp, vp, vp, dbl, ci, ctypes.POINTER(fl_solve_info), vp]
    L.fl_mg_solve.restype = ci
    L.fl_mg_last_error.argtypes = [vp]
    L.fl_mg_last_error.restype = ctypes.c_char_p
    L.fl_mg_destroy.argtypes = [vp]
    L.fl_mg_destroy.restype = None
    L.fl_patches.argtypes = [vp, dbl, ci, vp, vp, vp]
    L.fl_patches.restype = ci
    L.fl_lp_create.argtypes = [ctypes.POINTER(vp), vp, dbl, ci, ci, ctypes.c_uint64]
    L.fl_lp_create.restype = ci
    for nm, rt in (("fl_lp_num_params", i64), ("fl_lp_num_features", ci), ("fl_lp_num_samples", i64)):
        getattr(L, nm).argtypes = [vp]
        getattr(L, nm).restype = rt
    L.fl_lp_get_params.argtypes = [vp, vp]
    L.fl_lp_get_params.restype = ci
    L.fl_lp_set_params.argtypes = [vp, vp]
    L.fl_lp_set_params.restype = ci
    L.fl_lp_stencil.argtypes = [vp, vp]
    L.fl_lp_stencil.restype = ci
    L.fl_lp_bind.argtypes = [vp, vp, i64, vp]
    L.fl_lp_bind.restype = ci
    L.fl_lp_features.argtypes = [vp, vp, vp, vp, vp]
    L.fl_lp_features.restype = ci
    L.fl_lp_apply.argtypes = [vp, vp, vp, vp]
    L.fl_lp_apply.restype = ci
    L.fl_lp_loss_grad.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    L.fl_lp_loss_grad.restype = ci
    L.fl_lp_add_pairs.argtypes = [vp, vp, i64, vp, i64, ci, vp]
    L.fl_lp_add_pairs.restype = ci
    L.fl_lp_collect.argtypes = [vp, vp, i64, vp, ci, vp, vp]
    L.fl_lp_collect.restype = ci
    L.fl_lp_collect_noise.argtypes = [vp, vp, i64, ci, ci, vp, ctypes.c_uint64, vp]
    L.fl_lp_collect_noise.restype = ci
    L.fl_lp_train.argtypes = [vp, ci, i64, ctypes.c_float, ctypes.c_uint64, vp, vp]
    L.fl_lp_train.restype = ci
    L.fl_lp_last_error.argtypes = [vp]
    L.fl_lp_last_error.restype = ctypes.c_char_p
    L.fl_lp_destroy.argtypes = [vp]
    L.fl_lp_destroy.restype = None
    L.fl_fcg_solve.argtypes = [vp, i64, vp, i64, vp, vp, vp, vp, dbl, ci, ctypes.POINTER(fl_fcg_info), vp]
    L.fl_fcg_solve.restype = ci
    _ = i32
    _lib = L
    return L


def _check(code, handle=None):
    if code != FL_OK:
        msg = lib().fl_last_error(handle).decode(errors="replace")
        raise FlError(code, msg)


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


# ----------------------------------------------------------- C-named calls --
def fl_default_options():
    o = fl_options()
    lib().fl_default_options(ctypes.byref(o))
    return o


def fl_create(vertices, cells, dof_mode=FL_DOF_INTERIOR, options=None):
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    C = np.ascontiguousarray(cells, dtype=np.int32)
    h = ctypes.c_void_p()
    opt = options if options is not None else fl_default_options()
    r = lib().fl_create(ctypes.byref(h), V.shape[1], V.shape[0], V.ctypes.data, C.shape[0], C.ctypes.data, dof_mode,
                        ctypes.byref(opt))
    _check(r, None)
    return h


def fl_create_sector(vertices, cells, K, options=None):
    """Handle of the symmetry-reduced problem on the K rotated copies of a sector mesh."""
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    C = np.ascontiguousarray(cells, dtype=np.int32)
    h = ctypes.c_void_p()
    opt = options if options is not None else fl_default_options()
    _check(lib().fl_create_sector(ctypes.byref(h), V.shape[0], V.ctypes.data, C.shape[0], C.ctypes.data, K,
                                  ctypes.byref(opt)), None)
    return h


def fl_destroy(h):
    lib().fl_destroy(h)


def fl_num_dofs(h, s):
    n = ctypes.c_int64()
    _check(lib().fl_num_dofs(h, s, ctypes.byref(n)), h)
    return n.value


def fl_dof_vertices(h, s):
    out = np.empty(fl_num_dofs(h, s), dtype=np.int32)
    _check(lib().fl_dof_vertices(h, s, out.ctypes.data), h)
    return out


def fl_assemble(h, s, precision, A, stream=None):
    """A: float64 CUDA tensor [n, lda] (row-major, contiguous rows)."""
    assert A.dtype.is_floating_point and A.element_size() == 8 and A.is_cuda and A.stride(1) == 1
    _check(lib().fl_assemble(h, s, precision, _ptr(A), A.stride(0), _stream(stream)), h)


def fl_tune_assemble(h, s, A, reps=5, stream=None):
    """Sweep the float64-mode far-kernel launch variants on A's mesh (A as for fl_assemble);
    returns (best variant, its median far-stage ms) and records it in the tuning table."""
    v = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    _check(lib().fl_tune_assemble(h, s, _ptr(A), A.stride(0), reps, ctypes.byref(v), ctypes.byref(ms),
                                  _stream(stream)), h)
    return v.value, ms.value


def fl_set_far_variant(h, variant):
    _check(lib().fl_set_far_variant(h, variant), h)


def fl_assemble_nearfield_csr(h, s, precision, stream=None):
    """(rowptr int32 [n+1], col int32 [nnz], val float64 [nnz]) device tensors of the
    near-field part N of A = N + F."""
    import torch

    nnz = ctypes.c_int64(0)
    _check(lib().fl_assemble_nearfield_csr(h, s, precision, ctypes.byref(nnz), None, None, None, _stream(stream)), h)
    n = fl_num_dofs(h, s)
    rowptr = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(max(1, nnz.value), dtype=torch.int32, device="cuda")
    val = torch.empty(max(1, nnz.value), dtype=torch.float64, device="cuda")
    _check(lib().fl_assemble_nearfield_csr(h, s, precision, ctypes.byref(nnz), _ptr(rowptr), _ptr(col), _ptr(val),
                                           _stream(stream)), h)
    return rowptr, col[:nnz.value], val[:nnz.value]


def fl_load_vector(h, s, f_nodal, b, stream=None):
    """b: float64 CUDA tensor [n, nrhs]; f_nodal: None (f = 1) or float64 CUDA [n_vertices, nrhs]."""
    nrhs = b.shape[1] if b.dim() == 2 else 1
    ldb = b.stride(0) if b.dim() == 2 else 1
    fp = _ptr(f_nodal) if f_nodal is not None else None
    _check(lib().fl_load_vector(h, s, fp, nrhs, _ptr(b), ldb, _stream(stream)), h)


def _ld(dtype, M):
    # leading dimension in entries: an FL_F32X2 entry is two float32 values
    return M.stride(0) // 2 if dtype == FL_F32X2 else M.stride(0)


def fl_matvec(dtype, A, X, Y, stream=None):
    """Y = A X; an FL_F32X2 matrix is a float32 tensor [n, 2 * lda] of (hi, lo) pairs."""
    n = A.shape[0]
    nrhs = X.shape[1] if X.dim() == 2 else 1
    ldx = X.stride(0) if X.dim() == 2 else 1
    ldy = Y.stride(0) if Y.dim() == 2 else 1
    _check(lib().fl_matvec(dtype, _ptr(A), _ld(dtype, A), n, nrhs, _ptr(X), ldx, _ptr(Y), ldy, _stream(stream)))


def fl_convert(A, dtype, out, stream=None):
    _check(lib().fl_convert(_ptr(A), A.stride(0), A.shape[0], dtype, _ptr(out), _ld(dtype, out), _stream(stream)))


def fl_heat_matrix(h, s, dt, A, H, stream=None):
    """H = M + dt A (H may be A)."""
    _check(lib().fl_heat_matrix(h, s, dt, _ptr(A), A.stride(0), _ptr(H), H.stride(0), _stream(stream)), h)


def fl_mass_apply(h, s, alpha, X, beta, B, Y, stream=None):
    """Y = alpha M X + beta B (X, B, Y float64 [n] or [n, nrhs]; B may be None when beta = 0)."""
    nrhs = X.shape[1] if X.dim() == 2 else 1
    ld = lambda T: (T.stride(0) if T.dim() == 2 else 1) if T is not None else 1  # noqa: E731
    _check(lib().fl_mass_apply(h, s, nrhs, alpha, _ptr(X), ld(X), beta, _ptr(B) if B is not None else None, ld(B),
                               _ptr(Y), ld(Y), _stream(stream)), h)


def _rule_points(k_cell, dim):
    return k_cell if dim == 1 else k_cell * k_cell


def fl_strong_form(h, s, u, k_cell, k_edge, k_near, S, stream=None):
    """S [n_cells, q] = (-Delta)^s u_h at the cell-rule points (u: n float64 DOF values)."""
    _check(lib().fl_strong_form(h, s, _ptr(u), k_cell, k_edge, k_near, _ptr(S), _stream(stream)), h)


def fl_br_indicators(h, s, u, f_nodal, k_cell, k_edge, k_near, eta, S=None, stream=None):
    """eta [n] = BR indicators; f_nodal None (f = 1) or [n_vertices]; S optional [n_cells, q]."""
    _check(lib().fl_br_indicators(h, s, _ptr(u), _ptr(f_nodal) if f_nodal is not None else None, k_cell, k_edge,
                                  k_near, _ptr(eta), _ptr(S) if S is not None else None, _stream(stream)), h)


def fl_mark_max(h, s, eta, theta, dof_marks=None, cell_marks=None, stream=None):
    """Maximum marking into uint8 tensors dof_marks [n] and/or cell_marks [n_cells]."""
    _check(lib().fl_mark_max(h, s, _ptr(eta), theta, _ptr(dof_marks) if dof_marks is not None else None,
                             _ptr(cell_marks) if cell_marks is not None else None, _stream(stream)), h)


def fl_refine(vertices, cells, cell_marks):
    """Conforming refinement of the marked cells (host arrays): returns (vertices, cells)."""
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    C = np.ascontiguousarray(cells, dtype=np.int32)
    M = np.ascontiguousarray(cell_marks, dtype=np.uint8)
    if M.shape != (C.shape[0],):
        raise ValueError("one mark per cell")
    dim = V.shape[1]
    cap_v, cap_c = V.shape[0] + 3 * C.shape[0], 4 * C.shape[0]
    Vo = np.empty((cap_v, dim), dtype=np.float64)
    Co = np.empty((cap_c, dim + 1), dtype=np.int32)
    nv, nc = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().fl_refine(dim, V.shape[0], V.ctypes.data, C.shape[0], C.ctypes.data, M.ctypes.data, cap_v, cap_c,
                           Vo.ctypes.data, Co.ctypes.data, ctypes.byref(nv), ctypes.byref(nc)), None)
    Vo = Vo[:nv.value].copy()
    return (Vo[:, 0] if np.asarray(vertices).ndim == 1 else Vo), Co[:nc.value].copy()


def fl_cluster_plan(h, s, eta=1.0, leaf=32):
    """Host-only cluster tree and partition: dict with perm [n], node [nodes, 4] (lo, hi, son0,
    son1), far [pairs, 2], near [pairs, 2] (int32 numpy arrays)."""
    sizes = (ctypes.c_int64 * 3)()
    _check(lib().fl_cluster_plan(h, s, eta, leaf, sizes, None, None, None, None), h)
    nn, nf, nr = sizes[0], sizes[1], sizes[2]
    n = fl_num_dofs(h, s)
    perm = np.zeros(n, dtype=np.int32)
    node = np.zeros((nn, 4), dtype=np.int32)
    far = np.zeros((nf, 2), dtype=np.int32)
    near = np.zeros((nr, 2), dtype=np.int32)
    _check(lib().fl_cluster_plan(h, s, eta, leaf, sizes, perm.ctypes.data, node.ctypes.data, far.ctypes.data,
                                 near.ctypes.data), h)
    return {"perm": perm, "node": node, "far": far, "near": near}


def fl_near_region_plan(h, s, dim, eta=1.0, leaf=32):
    """Host-only plan of the direct near-field assembly for a dim-dimensional mesh: dict with
    tiles (count), cell_perm [cells], ef_ptr [cells + 1], ef_fac, ef_cls [entries], fac_vert
    [table, dim], fac_normal [table, dim] (numpy arrays)."""
    sizes = (ctypes.c_int64 * 4)()
    _check(lib().fl_near_region_plan(h, s, eta, leaf, sizes, None, None, None, None, None, None), h)
    nt, ne, nfac, nc = sizes[0], sizes[1], sizes[2], sizes[3]
    out = {"tiles": nt, "cell_perm": np.zeros(nc, dtype=np.int32), "ef_ptr": np.zeros(nc + 1, dtype=np.int32),
           "ef_fac": np.zeros(ne, dtype=np.int32), "ef_cls": np.zeros(ne, dtype=np.int32),
           "fac_vert": np.zeros((nfac, dim), dtype=np.int32), "fac_normal": np.zeros((nfac, dim))}
    _check(lib().fl_near_region_plan(h, s, eta, leaf, sizes, out["cell_perm"].ctypes.data, out["ef_ptr"].ctypes.data,
                                     out["ef_fac"].ctypes.data, out["ef_cls"].ctypes.data,
                                     out["fac_vert"].ctypes.data, out["fac_normal"].ctypes.data), h)
    return out


def fl_near_region_tiles(h, s, eta=1.0, leaf=32):
    """Host-only tile list of the direct near-field assembly: (tiles [ntiles, 2] int32 (I, J),
    rowmask [ntiles] uint32) (numpy arrays)."""
    nt = ctypes.c_int64()
    _check(lib().fl_near_region_tiles(h, s, eta, leaf, ctypes.byref(nt), None, None), h)
    tiles = np.zeros((nt.value, 2), dtype=np.int32)
    rowmask = np.zeros(nt.value, dtype=np.uint32)
    _check(lib().fl_near_region_tiles(h, s, eta, leaf, ctypes.byref(nt), tiles.ctypes.data, rowmask.ctypes.data), h)
    return tiles, rowmask


def fl_strong_form_cluster_plan(h, s, eta=1.0, leaf=32, k_cell=3):
    """Host-only plan of the cluster strong form: dict with pgroup [points], gnode [groups],
    gf_ptr [groups + 1], gf_fac [entries], fac_vert [facets, 2] (numpy arrays)."""
    sizes = (ctypes.c_int64 * 4)()
    _check(lib().fl_strong_form_cluster_plan(h, s, eta, leaf, k_cell, sizes, None, None, None, None, None), h)
    npts, ng, ne, nfac = sizes[0], sizes[1], sizes[2], sizes[3]
    out = {"pgroup": np.zeros(npts, dtype=np.int32), "gnode": np.zeros(ng, dtype=np.int32),
           "gf_ptr": np.zeros(ng + 1, dtype=np.int64), "gf_fac": np.zeros(ne, dtype=np.int32),
           "fac_vert": np.zeros((nfac, 2), dtype=np.int32)}
    _check(lib().fl_strong_form_cluster_plan(h, s, eta, leaf, k_cell, sizes, out["pgroup"].ctypes.data,
                                             out["gnode"].ctypes.data, out["gf_ptr"].ctypes.data,
                                             out["gf_fac"].ctypes.data, out["fac_vert"].ctypes.data), h)
    return out


class HMatrix:
    """Cluster-method approximation of A^s on a mesh handle (Section 6); owns an fl_hmatrix."""

    def __init__(self, h, s, m=4, eta=1.0, leaf=32, stream=None):
        self.hm = ctypes.c_void_p()
        _check(lib().fl_hmatrix_create(h, s, m, eta, leaf, ctypes.byref(self.hm), _stream(stream)), h)
        self.n = fl_num_dofs(h, s)
        self.n_cells = fl_get_stats(h, s)["n_cells"]
        self.h, self.s = h, s

    def _check(self, r):
        if r != FL_OK:
            raise FlError(r, lib().fl_hmatrix_last_error(self.hm).decode(errors="replace"))

    def set_near(self, A, stream=None):
        self._check(lib().fl_hmatrix_set_near(self.hm, _ptr(A), A.stride(0), _stream(stream)))

    def assemble_near(self, precision="fp64", stream=None):
        """Near-field entries by local computations (no dense matrix); precision "fp64" or "mixed"."""
        prec = {"fp64": FL_FP64, "mixed": FL_MIXED}[precision]
        self._check(lib().fl_hmatrix_assemble_near(self.hm, prec, _stream(stream)))

    def get_near(self, stream=None):
        """The near field as (rowptr, col, val) CUDA tensors (int32, int32, float64)."""
        import torch

        nnz = ctypes.c_int64(0)
        self._check(lib().fl_hmatrix_get_near(self.hm, ctypes.byref(nnz), None, None, None, None))
        n = self.n
        rowptr = torch.empty(n + 1, dtype=torch.int32, device="cuda")
        col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device="cuda")
        val = torch.empty(max(nnz.value, 1), dtype=torch.float64, device="cuda")
        self._check(lib().fl_hmatrix_get_near(self.hm, ctypes.byref(nnz), _ptr(rowptr), _ptr(col), _ptr(val),
                                              _stream(stream)))
        return rowptr, col[: nnz.value], val[: nnz.value]

    def strong_form(self, u, k_cell=3, k_edge=4, k_near=16, stream=None):
        """(-Delta)^s u_h by the cluster method at the cell-rule points: [cells, k_cell^2] tensor."""
        import torch

        S = torch.empty(self.n_cells, k_cell * k_cell, dtype=torch.float64, device=u.device)
        self._check(lib().fl_hmatrix_strong_form(self.hm, _ptr(u), k_cell, k_edge, k_near, _ptr(S), _stream(stream)))
        return S

    def br_indicators(self, u, f=None, k_cell=3, k_edge=4, k_near=16, stream=None):
        """(eta [n], S [cells, k_cell^2]) with the cluster method's strong form."""
        import torch

        S = torch.empty(self.n_cells, k_cell * k_cell, dtype=torch.float64, device=u.device)
        eta = torch.empty(self.n, dtype=torch.float64, device=u.device)
        self._check(lib().fl_hmatrix_br_indicators(self.hm, _ptr(u), _ptr(f) if f is not None else None, k_cell,
                                                   k_edge, k_near, _ptr(eta), _ptr(S), _stream(stream)))
        return eta, S

    def near_info(self):
        v = (ctypes.c_int64 * 3)()
        self._check(lib().fl_hmatrix_near_info(self.hm, v))
        return dict(zip(["tiles", "tile_entries", "device_bytes"], list(v)))

    def matvec(self, x, y, stream=None):
        self._check(lib().fl_hmatrix_matvec(self.hm, _ptr(x), _ptr(y), _stream(stream)))

    def solve(self, b, tol=1e-8, maxit=10000, stream=None):
        """Jacobi-PCG with the H-matrix product: (u, fl_solve_info); ENOTCONV / ENOTSPD are
        reported in info.status rather than raised."""
        import torch

        o = fl_default_solve_opts()
        o.tol, o.maxit = tol, maxit
        info = fl_solve_info()
        u = torch.empty_like(b)
        r = lib().fl_hmatrix_solve(self.hm, _ptr(b), _ptr(u), ctypes.byref(o), ctypes.byref(info), _stream(stream))
        if r not in (FL_OK, FL_ENOTCONV, FL_ENOTSPD):
            self._check(r)
        return u, info

    def solve_shifted(self, b, alpha, beta, tol=1e-8, maxit=10000, u=None, stream=None):
        """(alpha M + beta A_H) u = b by Jacobi-PCG with the H-matrix product (M the P1 mass
        matrix): (u, fl_solve_info), ENOTCONV / ENOTSPD reported in info.status."""
        import torch

        o = fl_default_solve_opts()
        o.tol, o.maxit = tol, maxit
        info = fl_solve_info()
        u = torch.empty_like(b) if u is None else u
        r = lib().fl_hmatrix_solve_shifted(self.hm, alpha, beta, _ptr(b), _ptr(u), ctypes.byref(o),
                                           ctypes.byref(info), _stream(stream))
        if r not in (FL_OK, FL_ENOTCONV, FL_ENOTSPD):
            self._check(r)
        return u, info

    def heat_steps(self, dt, u0, F, steps, tol=1e-10, stream=None):
        """Implicit Euler for the fractional heat equation (Sections 2 and 5) with the cluster
        method: (M + dt A) u^{k+1} = M u^k + dt F, `steps` steps from u0 (F the load vector).
        Returns (u, list of fl_solve_info)."""
        import torch

        u = u0.clone()
        rhs = torch.empty_like(u0)
        infos = []
        for _ in range(steps):
            _check(lib().fl_mass_apply(self.h, self.s, 1, 1.0, _ptr(u), 1, dt, _ptr(F), 1, _ptr(rhs), 1,
                                       _stream(stream)), self.h)
            u, info = self.solve_shifted(rhs, 1.0, dt, tol=tol, stream=stream)
            if info.status != FL_OK:
                raise FlError(info.status, "heat step did not converge")
            infos.append(info)
        return u, infos

    def info(self):
        v = (ctypes.c_int64 * 6)()
        self._check(lib().fl_hmatrix_info(self.hm, v))
        return dict(zip(["nodes", "far_pairs", "near_pairs", "near_entries", "device_bytes", "depth"], list(v)))

    def close(self):
        if self.hm:
            lib().fl_hmatrix_destroy(self.hm)
            self.hm = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fl_default_solve_opts():
    o = fl_solve_opts()
    lib().fl_default_solve_opts(ctypes.byref(o))
    return o


def fl_solve(h, A, b, u, opts=None, stream=None):
    """Returns fl_solve_info; raises on FL_EINVAL / FL_ENOMEM / FL_ECUDA, not on FL_ENOTCONV / FL_ENOTSPD."""
    o = opts if opts is not None else fl_default_solve_opts()
    info = fl_solve_info()
    r = lib().fl_solve(h, A.shape[0], _ptr(A), A.stride(0), _ptr(b), _ptr(u), ctypes.byref(o), ctypes.byref(info),
                       _stream(stream))
    if r not in (FL_OK, FL_ENOTCONV, FL_ENOTSPD):
        _check(r, h)
    return info


def fl_get_stats(h, s):
    st = fl_stats()
    _check(lib().fl_get_stats(h, s, ctypes.byref(st)), h)
    return {k: getattr(st, k) for k, _ in fl_stats._fields_}


def fl_set_profiling(h, enable=True):
    """enable: False/0 off, True/1 every stage in sequence, 2 the far stage alone (schedule kept)."""
    _check(lib().fl_set_profiling(h, int(enable)), h)


def fl_stage_ms(h):
    out = (ctypes.c_double * len(STAGES))()
    _check(lib().fl_stage_ms(h, out), h)
    return dict(zip(STAGES, list(out)))


def fl_launch_count():
    return int(lib().fl_launch_count())


def fl_pool_trim():
    """Release the allocator's cached device and pinned host blocks; returns the bytes released."""
    return int(lib().fl_pool_trim())


def fl_pool_stats():
    v = [ctypes.c_int64() for _ in range(4)]
    lib().fl_pool_stats(*[ctypes.byref(x) for x in v])
    return {"cached_device_bytes": v[0].value, "cached_host_bytes": v[1].value, "hits": v[2].value,
            "misses": v[3].value}


def fl_matvec_f32_static(A32, x, y, stream=None):
    """y = A32 x without any device allocation (for callers that cannot allocate);
    n <= FL_STATIC_MAX_N.  A32: float32 CUDA [n, lda] with unit column stride; x, y:
    contiguous float64 CUDA vectors of length n.  Returns the status code (0 = FL_OK)
    instead of raising."""
    import torch

    n = A32.shape[0]
    if A32.dtype != torch.float32 or A32.dim() != 2 or A32.shape[1] != n or A32.stride(1) != 1:
        raise ValueError("A32 must be an n x n float32 matrix with unit column stride")
    for name, v in (("x", x), ("y", y)):
        if v.dtype != torch.float64 or v.dim() != 1 or v.shape[0] != n or not v.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 vector of length {n}")
    if not (A32.is_cuda and x.is_cuda and y.is_cuda):
        raise ValueError("A32, x and y must be CUDA tensors")
    return lib().fl_matvec_f32_static(_ptr(A32), A32.stride(0), n, _ptr(x), _ptr(y), _stream(stream))


def fl_split_bf16_bytes(n, nslices):
    return int(lib().fl_split_bf16_bytes(n, nslices))


def fl_split_bf16(A, nslices, S, dscale, stream=None):
    """A: float64 [n, lda]; S: CUDA tensor of at least fl_split_bf16_bytes(n, nslices) bytes
    (tiled layout, see fraclap.h); dscale: float64 [n]."""
    n = A.shape[0]
    assert S.numel() * S.element_size() >= fl_split_bf16_bytes(n, nslices)
    _check(lib().fl_split_bf16(_ptr(A), A.stride(0), n, nslices, _ptr(S), _ptr(dscale), _stream(stream)))


def split_bf16(A, nslices=2, stream=None):
    """Allocate and fill the slices of A: returns (S as a uint8 CUDA tensor, dscale)."""
    import torch

    n = A.shape[0]
    S = torch.empty(fl_split_bf16_bytes(n, nslices), dtype=torch.uint8, device=A.device)
    d = torch.empty(n, dtype=torch.float64, device=A.device)
    fl_split_bf16(A, nslices, S, d, stream)
    return S, d


def fl_matmul_bf16(S, n, nslices, X, Y, stream=None):
    """S from fl_split_bf16; X, Y: float32 CUDA tensors [nrhs, n] (one right-hand side per row)."""
    _check(lib().fl_matmul_bf16(_ptr(S), n, nslices, X.shape[0], _ptr(X), X.stride(0), _ptr(Y), Y.stride(0),
                                _stream(stream)))


def fl_default_batch_opts():
    o = fl_batch_opts()
    lib().fl_default_batch_opts(ctypes.byref(o))
    return o


def _batch_array(problems):
    arr = (fl_batch_problem * len(problems))()
    for k, q in enumerate(problems):
        A, S, B, U = q.get("A"), q["S"], q["B"], q.get("U")
        arr[k] = fl_batch_problem(A.shape[0] if A is not None else q["n"],
                                  A.data_ptr() if A is not None else None, A.stride(0) if A is not None else 0,
                                  S.data_ptr(), q["nslices"], q["dscale"].data_ptr() if "dscale" in q else None,
                                  B.shape[1], B.data_ptr(), B.stride(0), U.data_ptr() if U is not None else None,
                                  U.stride(0) if U is not None else 0)
    return arr


def fl_tune_batch(h, problems, reps=5):
    """Autotune the batched tensor-core product on these problems; returns (fl_batch_opts, ms)."""
    arr = _batch_array(problems)
    best = fl_batch_opts()
    ms = ctypes.c_double()
    _check(lib().fl_tune_batch(h, len(problems), arr, reps, ctypes.byref(best), ctypes.byref(ms)), h)
    return best, ms.value


def fl_tune_matvec(dtype, A, x, y, reps=5, stream=None):
    """Tune fl_matvec's blocks per SM on A (float64 or float32, n x n, row stride lda);
    x, y: [n] float64.  Returns (blocks per SM, ms)."""
    per_sm = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    _check(lib().fl_tune_matvec(dtype, _ptr(A), A.stride(0), A.shape[0], _ptr(x), _ptr(y), reps, ctypes.byref(per_sm),
                                ctypes.byref(ms), _stream(stream)))
    return per_sm.value, ms.value


def fl_tune_record(kernel, n, nrhs, nslices, p0, p1, ms):
    _check(lib().fl_tune_record(kernel.encode(), n, nrhs, nslices, p0, p1, ms))


def fl_tune_lookup(kernel, n, nrhs, nslices):
    """(p0, p1) or None."""
    a, b = ctypes.c_int(), ctypes.c_int()
    r = lib().fl_tune_lookup(kernel.encode(), n, nrhs, nslices, ctypes.byref(a), ctypes.byref(b))
    return (a.value, b.value) if r == FL_OK else None


def fl_tune_clear():
    lib().fl_tune_clear()


def fl_tune_count():
    return int(lib().fl_tune_count())


def fl_tune_save(path):
    _check(lib().fl_tune_save(os.fspath(path).encode()))


def fl_tune_load(path):
    _check(lib().fl_tune_load(os.fspath(path).encode()))


def fl_prolongation(fine, coarse, s):
    """Host CSR (rowptr, col, val) of the prolongation from coarse to fine DOFs."""
    nnz = ctypes.c_int64()
    _check(lib().fl_prolongation(fine, coarse, s, ctypes.byref(nnz), None, None, None), fine)
    n = fl_num_dofs(fine, s)
    ptr = np.zeros(n + 1, dtype=np.int32)
    col = np.zeros(nnz.value, dtype=np.int32)
    val = np.zeros(nnz.value, dtype=np.float64)
    _check(lib().fl_prolongation(fine, coarse, s, ctypes.byref(nnz), ptr.ctypes.data, col.ctypes.data,
                                 val.ctypes.data), fine)
    return ptr, col, val


class Multigrid:
    """Galerkin V-cycle hierarchy (fl_mg_*) on a finest float64 operator A (kept alive here)."""

    def __init__(self, A):
        self.A = A
        self.m = ctypes.c_void_p()
        r = lib().fl_mg_create(ctypes.byref(self.m), _ptr(A), A.stride(0), A.shape[0])
        if r != FL_OK:
            raise FlError(r, "fl_mg_create")

    def _check(self, r):
        if r != FL_OK:
            raise FlError(r, lib().fl_mg_last_error(self.m).decode(errors="replace"))

    def add_level(self, ptr, col, val, nc, stream=None):
        ptr = np.ascontiguousarray(ptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        self._check(lib().fl_mg_add_level(self.m, nc, len(col), ptr.ctypes.data, col.ctypes.data, val.ctypes.data,
                                          _stream(stream)))

    def setup(self, nu=2, stream=None):
        self._check(lib().fl_mg_setup(self.m, nu, _stream(stream)))

    def level(self, k):
        """(n, device pointer, lda) of level k."""
        n, p, ld = ctypes.c_int64(), ctypes.c_void_p(), ctypes.c_int64()
        self._check(lib().fl_mg_level(self.m, k, ctypes.byref(n), ctypes.byref(p), ctypes.byref(ld)))
        return n.value, p.value, ld.value

    def level_matrix(self, k, stream=None):
        """A copy of level k's float64 operator as a CUDA tensor."""
        import torch

        n = self.level(k)[0]
        out = torch.empty((n, n), dtype=torch.float64, device="cuda")
        self._check(lib().fl_mg_level_copy(self.m, k, _ptr(out), n, _stream(stream)))
        return out

    def omega(self, k):
        w = ctypes.c_float()
        self._check(lib().fl_mg_omega(self.m, k, ctypes.byref(w)))
        return w.value

    def vcycle(self, r32, z32, stream=None):
        self._check(lib().fl_mg_vcycle(self.m, _ptr(r32), _ptr(z32), _stream(stream)))

    def solve(self, b, u, tol=1e-8, maxit=1000, stream=None):
        info = fl_solve_info()
        r = lib().fl_mg_solve(self.m, _ptr(b), _ptr(u), tol, maxit, ctypes.byref(info), _stream(stream))
        if r not in (FL_OK, FL_ENOTCONV, FL_ENOTSPD):
            self._check(r)
        return info

    def close(self):
        if self.m:
            lib().fl_mg_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fl_patches(h, s, K=12):
    """(nbr [n, K] int32, h [n] float64, hop [n] int32) of the mesh's DOFs (host)."""
    n = fl_num_dofs(h, s)
    nbr = np.zeros((n, K), dtype=np.int32)
    hl = np.zeros(n, dtype=np.float64)
    hop = np.zeros(n, dtype=np.int32)
    _check(lib().fl_patches(h, s, K, nbr.ctypes.data, hl.ctypes.data, hop.ctypes.data), h)
    return nbr, hl, hop


class LearnedPreconditioner:
    """fl_lp_* handle: patch-MLP preconditioner for one mesh (which must stay alive)."""

    def __init__(self, mesh_handle, s, seed=1, K=12, hidden=64):
        self.m = ctypes.c_void_p()
        r = lib().fl_lp_create(ctypes.byref(self.m), mesh_handle, s, K, hidden, seed)
        if r != FL_OK:
            raise FlError(r, "fl_lp_create")
        self.n = fl_num_dofs(mesh_handle, s)
        self.nw = int(lib().fl_lp_num_params(self.m))
        self.F = int(lib().fl_lp_num_features(self.m))

    def _check(self, r):
        if r != FL_OK:
            raise FlError(r, lib().fl_lp_last_error(self.m).decode(errors="replace"))

    def params(self):
        out = np.zeros(self.nw, dtype=np.float32)
        self._check(lib().fl_lp_get_params(self.m, out.ctypes.data))
        return out

    def set_params(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == self.nw
        self._check(lib().fl_lp_set_params(self.m, w.ctypes.data))

    def stencil(self):
        out = np.zeros((self.n, 13), dtype=np.float32)
        self._check(lib().fl_lp_stencil(self.m, out.ctypes.data))
        return out

    def bind(self, A, stream=None):
        self._check(lib().fl_lp_bind(self.m, _ptr(A), A.stride(0), _stream(stream)))

    def features(self, r, stream=None):
        import torch

        X = torch.empty((self.n, self.F), dtype=torch.float32, device="cuda")
        sig = torch.empty(self.n, dtype=torch.float32, device="cuda")
        self._check(lib().fl_lp_features(self.m, _ptr(r), _ptr(X), _ptr(sig), _stream(stream)))
        return X, sig

    def apply(self, r, z, stream=None):
        self._check(lib().fl_lp_apply(self.m, _ptr(r), _ptr(z), _stream(stream)))

    def loss_grad(self, X, T, stream=None):
        loss = ctypes.c_float()
        g = np.zeros(self.nw, dtype=np.float32)
        self._check(lib().fl_lp_loss_grad(self.m, X.shape[0], _ptr(X), _ptr(T), ctypes.byref(loss), g.ctypes.data,
                                          _stream(stream)))
        return loss.value, g

    def add_pairs(self, A, E, stream=None):
        """E: float64 [count, n] (one error vector per row)."""
        self._check(lib().fl_lp_add_pairs(self.m, _ptr(A), A.stride(0), _ptr(E), E.stride(0), E.shape[0],
                                          _stream(stream)))

    def collect(self, A, b, ks, stream=None):
        k = np.ascontiguousarray(ks, dtype=np.int32)
        self._check(lib().fl_lp_collect(self.m, _ptr(A), A.stride(0), _ptr(b), len(k), k.ctypes.data,
                                        _stream(stream)))

    def collect_noise(self, A, count, ks, seed=20170813, stream=None):
        k = np.ascontiguousarray(ks, dtype=np.int32)
        self._check(lib().fl_lp_collect_noise(self.m, _ptr(A), A.stride(0), count, len(k), k.ctypes.data, seed,
                                              _stream(stream)))

    def num_samples(self):
        return int(lib().fl_lp_num_samples(self.m))

    def train(self, steps, batch=4096, lr=1e-3, seed=7, stream=None):
        loss = ctypes.c_float()
        self._check(lib().fl_lp_train(self.m, steps, batch, lr, seed, ctypes.byref(loss), _stream(stream)))
        return loss.value

    def close(self):
        if self.m:
            lib().fl_lp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fl_fcg_solve(h, A, b, u, lp=None, mg=None, tol=1e-8, maxit=2000, stream=None):
    """Flexible CG; returns fl_fcg_info (raises on argument / device errors)."""
    info = fl_fcg_info()
    r = lib().fl_fcg_solve(h, A.shape[0], _ptr(A), A.stride(0), _ptr(b), _ptr(u), lp.m if lp is not None else None,
                           mg.m if mg is not None else None, tol, maxit, ctypes.byref(info), _stream(stream))
    if r not in (FL_OK, FL_ENOTCONV, FL_ENOTSPD):
        _check(r, h)
    return info


def fl_batch_solve(h, problems, opts=None, stream=None):
    """problems: list of dicts with keys A (float64 [n, n]), S, nslices, dscale, B (float64 [n, nrhs]),
    U (float64 [n, nrhs], overwritten).  Returns (status, fl_batch_info, rel_residuals, statuses);
    raises on FL_EINVAL / FL_ENOMEM / FL_ECUDA / FL_ETIMEOUT / FL_ENOTIMPL."""
    arr = (fl_batch_problem * len(problems))()
    total = 0
    for k, q in enumerate(problems):
        A, S, B, U = q["A"], q["S"], q["B"], q["U"]
        arr[k] = fl_batch_problem(A.shape[0], A.data_ptr(), A.stride(0), S.data_ptr(), q["nslices"],
                                  q["dscale"].data_ptr(), B.shape[1], B.data_ptr(), B.stride(0), U.data_ptr(),
                                  U.stride(0))
        total += B.shape[1]
    o = opts if opts is not None else fl_default_batch_opts()
    info = fl_batch_info()
    rel = np.zeros(total, dtype=np.float64)
    st = np.zeros(total, dtype=np.int32)
    r = lib().fl_batch_solve(h, len(problems), arr, ctypes.byref(o), ctypes.byref(info), rel.ctypes.data,
                             st.ctypes.data, _stream(stream))
    if r not in (FL_OK, FL_ENOTCONV, FL_ENOTSPD):
        _check(r, h)
    return r, info, rel, st


# ------------------------------------------------------------- convenience --
class Mesh:
    """Owns one fl_handle.  Orders and the DOF rule are fixed at creation."""

    def __init__(self, vertices, cells, dof_mode="interior", k_far=4, k_near=6, k_touch=8, k_bnd=8, regional=False,
                 k_vertex=6, far_f64_pipe=False):
        o = fl_default_options()
        o.k_far, o.k_near, o.k_touch, o.k_bnd, o.regional = k_far, k_near, k_touch, k_bnd, int(regional)
        o.k_vertex = k_vertex
        o.far_f64_pipe = int(far_f64_pipe)
        self.h = fl_create(vertices, cells, FL_DOF_PAPER if dof_mode == "paper" else FL_DOF_INTERIOR, o)
        self.dim = 1 if np.asarray(vertices).ndim == 1 else np.asarray(vertices).shape[1]

    @classmethod
    def sector(cls, vertices, cells, K, k_far=4, k_near=6, k_touch=8, k_bnd=8, k_vertex=6, far_f64_pipe=False):
        """The symmetry-reduced problem (Section 7): the sector mesh's K rotated copies, one
        unknown per orbit; assemble / load_vector / solve then work on the reduced system
        (load_vector takes f on the sector's vertices)."""
        m = cls.__new__(cls)
        o = fl_default_options()
        o.k_far, o.k_near, o.k_touch, o.k_bnd, o.k_vertex = k_far, k_near, k_touch, k_bnd, k_vertex
        o.far_f64_pipe = int(far_f64_pipe)
        m.h = fl_create_sector(vertices, cells, K, o)
        m.dim = 2
        return m

    def close(self):
        if self.h:
            fl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_dofs(self, s):
        return fl_num_dofs(self.h, s)

    def dof_vertices(self, s):
        return fl_dof_vertices(self.h, s)

    def nearfield_csr(self, s, precision="fp64", stream=None):
        return fl_assemble_nearfield_csr(self.h, s, FL_MIXED if precision == "mixed" else FL_FP64, stream)

    def assemble(self, s, precision="fp64", out=None, stream=None):
        import torch

        n = self.num_dofs(s)
        A = out if out is not None else torch.empty((n, n), dtype=torch.float64, device="cuda")
        fl_assemble(self.h, s, FL_MIXED if precision == "mixed" else FL_FP64, A, stream)
        return A

    def load_vector(self, s, f_nodal=None, stream=None):
        import torch

        n = self.num_dofs(s)
        nrhs = 1 if f_nodal is None else (f_nodal.shape[1] if f_nodal.dim() == 2 else 1)
        b = torch.empty((n, nrhs), dtype=torch.float64, device="cuda")
        f = None if f_nodal is None else f_nodal.reshape(f_nodal.shape[0], nrhs).contiguous()
        fl_load_vector(self.h, s, f, b, stream)
        return b[:, 0] if nrhs == 1 else b

    def solve(self, A, b, tol=1e-8, maxit=10000, A_lo=None, inner_tol=1e-4, inner_maxit=2000, stream=None):
        import torch

        o = fl_default_solve_opts()
        o.tol, o.maxit = tol, maxit
        if A_lo is not None:
            o.inner_dtype = FL_F32 if A_lo.dtype == torch.float32 else FL_BF16
            o.A_lo_dev = A_lo.data_ptr()
            o.ld_lo = A_lo.stride(0)
            o.inner_tol, o.inner_maxit = inner_tol, inner_maxit
        u = torch.empty_like(b)
        info = fl_solve(self.h, A, b, u, o, stream)
        return u, info

    def strong_form(self, s, u, k_cell=3, k_edge=4, k_near=16, stream=None):
        """(-Delta)^s u_h at the cell-rule points: float64 tensor [n_cells, q] (Lemma 4.1)."""
        import torch

        nc = fl_get_stats(self.h, s)["n_cells"]
        S = torch.empty((nc, _rule_points(k_cell, self.dim)), dtype=torch.float64, device=u.device)
        fl_strong_form(self.h, s, u, k_cell, k_edge, k_near, S, stream)
        return S

    def br_indicators(self, s, u, f_nodal=None, k_cell=3, k_edge=4, k_near=16, return_S=False, stream=None):
        """Babuska-Rheinboldt indicators eta [n] (and the strong form with return_S)."""
        import torch

        eta = torch.empty(self.num_dofs(s), dtype=torch.float64, device=u.device)
        S = None
        if return_S:
            nc = fl_get_stats(self.h, s)["n_cells"]
            S = torch.empty((nc, _rule_points(k_cell, self.dim)), dtype=torch.float64, device=u.device)
        fl_br_indicators(self.h, s, u, f_nodal, k_cell, k_edge, k_near, eta, S, stream)
        return (eta, S) if return_S else eta

    def mark_max(self, s, eta, theta=0.8, stream=None):
        """Maximum marking: (dof_marks [n], cell_marks [n_cells]) as uint8 tensors."""
        import torch

        nc = fl_get_stats(self.h, s)["n_cells"]
        dm = torch.empty(eta.shape[0], dtype=torch.uint8, device=eta.device)
        cm = torch.empty(nc, dtype=torch.uint8, device=eta.device)
        fl_mark_max(self.h, s, eta, theta, dm, cm, stream)
        return dm, cm

    def heat_steps(self, A, s, dt, u0, F, steps, tol=1e-10, stream=None):
        """Implicit Euler for the fractional heat equation (Sections 2 and 5): from u0, `steps`
        solves of (M + dt A) u^{k+1} = M u^k + dt F by Jacobi-PCG.  Returns (u, [fl_solve_info])."""
        import torch

        H = torch.empty_like(A)
        fl_heat_matrix(self.h, s, dt, A, H, stream)
        u = u0.clone()
        rhs = torch.empty_like(u0)
        o = fl_default_solve_opts()
        o.tol = tol
        infos = []
        for _ in range(steps):
            fl_mass_apply(self.h, s, 1.0, u, dt, F, rhs, stream)
            infos.append(fl_solve(self.h, H, rhs, u, o, stream))
        return u, infos


def adaptive_loop(vertices, cells, s, steps, theta=0.8, f_nodal=None, tol=1e-10, k_cell=3, k_edge=4, k_near=16,
                  max_dofs=None, dof_mode="interior", timings=False, cluster=None):
    """The adaptive loop of Section 7.  Per step: assemble A^s (float64) and b, solve A u = b
    (Jacobi-PCG), compute the BR indicators, mark with the maximum strategy (threshold theta) and
    refine the marked patches (newest-vertex bisection with closure).  f_nodal: None (f = 1) or
    a function of the vertex coordinates [nv, d] returning nodal values.  Stops after `steps`
    solves or once n exceeds max_dofs.  Returns one dict per step (host arrays: vertices,
    cells, u, eta, dof_marks, cell_marks; n, iterations; with timings, the milliseconds of
    assembly, solve and indicators by CUDA events).

    cluster: None (dense matrix, direct strong form) or a dict of HMatrix parameters (m, eta,
    leaf): every step then uses the cluster method of Section 6 throughout -- the near field by
    local computations, Jacobi-PCG on the H-matrix, the indicators from the cluster strong form --
    and forms no dense matrix."""
    import torch

    if cluster is not None:
        return _adaptive_loop_cluster(vertices, cells, s, steps, theta, f_nodal, tol, k_cell, k_edge, k_near,
                                      max_dofs, dof_mode, timings, dict(cluster))

    V = np.asarray(vertices, dtype=np.float64)
    C = np.asarray(cells, dtype=np.int32)
    out = []
    for _ in range(steps):
        mesh = Mesh(V, C, dof_mode=dof_mode)
        try:
            n = mesh.num_dofs(s)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if timings else None
            fv = None
            if f_nodal is not None:
                fv = torch.as_tensor(np.ascontiguousarray(f_nodal(V), dtype=np.float64), device="cuda")
            if ev:
                ev[0].record()
            A = mesh.assemble(s)
            b = mesh.load_vector(s, fv)
            if ev:
                ev[1].record()
            u, info = mesh.solve(A, b, tol=tol)
            if ev:
                ev[2].record()
            eta = mesh.br_indicators(s, u, fv, k_cell, k_edge, k_near)
            if ev:
                ev[3].record()
            dm, cm = mesh.mark_max(s, eta, theta)
            torch.cuda.synchronize()
            rec = {"vertices": V, "cells": C, "n": n, "u": u.cpu().numpy(), "eta": eta.cpu().numpy(),
                   "dof_marks": dm.cpu().numpy(), "cell_marks": cm.cpu().numpy(), "iterations": info.iterations}
            if ev:
                rec["ms"] = {"assemble": ev[0].elapsed_time(ev[1]), "solve": ev[1].elapsed_time(ev[2]),
                             "indicators": ev[2].elapsed_time(ev[3])}
            out.append(rec)
        finally:
            mesh.close()
        if max_dofs is not None and n >= max_dofs:
            break
        V, C = fl_refine(V, C, rec["cell_marks"])
    return out


def _adaptive_loop_cluster(vertices, cells, s, steps, theta, f_nodal, tol, k_cell, k_edge, k_near, max_dofs, dof_mode,
                           timings, cp):
    import torch

    V = np.asarray(vertices, dtype=np.float64)
    C = np.asarray(cells, dtype=np.int32)
    out = []
    for _ in range(steps):
        mesh = Mesh(V, C, dof_mode=dof_mode)
        H = None
        try:
            n = mesh.num_dofs(s)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if timings else None
            fv = None
            if f_nodal is not None:
                fv = torch.as_tensor(np.ascontiguousarray(f_nodal(V), dtype=np.float64), device="cuda")
            if ev:
                ev[0].record()
            H = HMatrix(mesh.h, s, m=cp.get("m", 4), eta=cp.get("eta", 1.0), leaf=cp.get("leaf", 32))
            H.assemble_near()
            b = mesh.load_vector(s, fv)
            if ev:
                ev[1].record()
            u, info = H.solve(b, tol=tol)
            if info.status != FL_OK:
                raise FlError(info.status, "H-matrix solve did not converge")
            if ev:
                ev[2].record()
            eta, _ = H.br_indicators(u, fv, k_cell, k_edge, k_near)
            if ev:
                ev[3].record()
            dm, cm = mesh.mark_max(s, eta, theta)
            torch.cuda.synchronize()
            rec = {"vertices": V, "cells": C, "n": n, "u": u.cpu().numpy(), "eta": eta.cpu().numpy(),
                   "dof_marks": dm.cpu().numpy(), "cell_marks": cm.cpu().numpy(), "iterations": info.iterations}
            if ev:
                rec["ms"] = {"assemble": ev[0].elapsed_time(ev[1]), "solve": ev[1].elapsed_time(ev[2]),
                             "indicators": ev[2].elapsed_time(ev[3])}
            out.append(rec)
        finally:
            if H is not None:
                H.close()
            mesh.close()
        if max_dofs is not None and n >= max_dofs:
            break
        V, C = fl_refine(V, C, rec["cell_marks"])
    return out
