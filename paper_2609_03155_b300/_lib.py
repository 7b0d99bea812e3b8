"""ctypes binding of libdpg.so (include/dpg.h): argument marshalling only.

Every function here forwards to the C ABI of the same name; device buffers
are torch CUDA tensors passed by data pointer, streams are torch streams
passed by handle.  There is no fallback: if the shared library is missing or
fails to load, importing the functions raises.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdpg.so")

DPG_OK = 0
ERRORS = {-1: "DPG_ERR_ARG", -2: "DPG_ERR_MESH", -3: "DPG_ERR_NOMEM", -4: "DPG_ERR_NOT_HPD",
          -5: "DPG_ERR_NOT_CONVERGED", -6: "DPG_ERR_TIMEOUT", -7: "DPG_ERR_CUDA", -8: "DPG_ERR_STATE",
          -9: "DPG_ERR_UNSUPPORTED"}
DPG_BC_NONE, DPG_BC_DIRICHLET, DPG_BC_ROBIN = 0, 1, 2
DPG_PASS_ASSEMBLE = 0
DPG_CG_FP64, DPG_CG_IR_FP32, DPG_CG_JACOBI, DPG_CG_BLOCK_JACOBI = 0, 1, 2, 4
DPG_PREC_FP64, DPG_PREC_TF32, DPG_PREC_3XTF32 = 0, 1, 2
DPG_CG_X0 = 8
DPG_CG_HALF = 16
DPG_CG_IR_V64 = 32
DPG_CG_DW = 64
DPG_CG_EBE = 128
DPG_CG_RELIABLE = 256
DPG_CG_EBE_BULK = 512
DPG_FLAG_ADJOINT = 1
DPG_FLAG_STREAM = 2
DPG_FACTOR_FP64, DPG_FACTOR_TC_SPLIT = 0, 1


class dpg_complex(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class dpg_robin_group(C.Structure):
    _fields_ = [("zinv_re", C.c_double), ("zinv_im", C.c_double), ("port", C.c_int32), ("m", C.c_int32),
                ("n", C.c_int32), ("a", C.c_double), ("b", C.c_double), ("eps_re", C.c_double),
                ("eps_im", C.c_double), ("mu_re", C.c_double), ("mu_im", C.c_double)]


class dpg_dirichlet_group(C.Structure):
    _fields_ = [("kind", C.c_int32), ("m", C.c_int32), ("n", C.c_int32), ("a", C.c_double), ("b", C.c_double),
                ("eps_re", C.c_double), ("eps_im", C.c_double), ("mu_re", C.c_double), ("mu_im", C.c_double)]


class dpg_mesh_desc(C.Structure):
    _fields_ = [("n_vert", C.c_int32), ("vert", C.c_void_p), ("n_elem", C.c_int32), ("elem", C.c_void_p),
                ("elem_p", C.c_void_p), ("elem_eps", C.c_void_p), ("elem_mu", C.c_void_p),
                ("face_bc", C.c_void_p), ("face_grp", C.c_void_p), ("n_robin", C.c_int32),
                ("robin", C.POINTER(dpg_robin_group)), ("n_dirichlet", C.c_int32),
                ("dirichlet", C.POINTER(dpg_dirichlet_group))]


class dpg_params(C.Structure):
    _fields_ = [("omega", C.c_double), ("alpha", C.c_double), ("dp", C.c_int32), ("precision", C.c_int32),
                ("chunk", C.c_int32), ("flags", C.c_int32)]


class dpg_cg_report(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("outer", C.c_int32), ("rel_residual", C.c_double),
                ("ms", C.c_double), ("converged", C.c_int32), ("reserved", C.c_int32)]


class dpg_timing(C.Structure):
    _fields_ = [("factor_ms", C.c_double), ("factor_launches", C.c_int64), ("factor_elements", C.c_int64),
                ("cg_ms", C.c_double), ("cg_iterations", C.c_int64), ("kernel_launches", C.c_int64),
                ("factor_ms_real", C.c_double), ("factor_elements_real", C.c_int64),
                ("cg_kernel_ms", C.c_double), ("cg_kernel_launches", C.c_int64),
                ("cg_kernel_iterations", C.c_int64)]


class DPGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libdpg.so once; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2609_03155_b300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    L.dpg_setup_mesh.argtypes = [C.POINTER(vp), C.POINTER(dpg_mesh_desc), C.POINTER(dpg_params), vp]
    L.dpg_element_batch.argtypes = [vp, i32, vp]
    L.dpg_assemble.argtypes = [vp, vp]
    L.dpg_cg_solve.argtypes = [vp, i32, dbl, dbl, i32, dbl, vp, vp, C.POINTER(dpg_cg_report), vp]
    L.dpg_estimate.argtypes = [vp, vp, vp, vp, C.POINTER(dbl), vp]
    L.dpg_estimate_noalloc.argtypes = [vp, vp, vp, vp, C.POINTER(dbl), vp]
    L.dpg_sizes.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                            C.POINTER(i32)]
    L.dpg_trace_map.argtypes = [vp, vp, vp]
    L.dpg_element_layout.argtypes = [vp, vp, vp, vp]
    L.dpg_tc_gemm.argtypes = [i32, i32, i32, i32, vp, vp, vp, i32]
    L.dpg_set_graph.argtypes = [vp, i32]
    L.dpg_set_wait_limit.argtypes = [vp, i64, i32]
    L.dpg_set_factor_arith.argtypes = [vp, i32]
    L.dpg_set_bucketed.argtypes = [vp, i32]
    L.dpg_set_estimator_store.argtypes = [vp, i32]
    L.dpg_factor_balance.argtypes = [vp, C.POINTER(dbl), C.POINTER(dbl), C.POINTER(i64)]
    L.dpg_estimate_clamped.argtypes = [vp, C.POINTER(i32)]
    L.dpg_mark_fraction.argtypes = [vp, vp, dbl, dbl, i32, vp, vp]
    L.dpg_factor_check.argtypes = [i32, i32, i32, i32, i32, i32, vp, vp, C.POINTER(i32)]
    L.dpg_power.argtypes = [vp, vp, vp, vp, vp]
    L.dpg_autotune.argtypes = [vp, dbl, vp, vp, vp]
    L.dpg_group_info.argtypes = [vp, vp, vp, vp, vp]
    L.dpg_element_dump.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp, vp]
    L.dpg_csr_copy.argtypes = [vp, vp, vp, vp, vp, vp]
    L.dpg_probe_peaks.argtypes = [C.POINTER(dbl), C.POINTER(dbl), vp]
    L.dpg_update_elements.argtypes = [vp, vp, vp, vp, vp]
    L.dpg_grad_eps.argtypes = [vp, vp, vp, C.POINTER(dbl), vp, vp, i32, dbl, i32, vp]
    L.dpg_timing_enable.argtypes = [vp, i32]
    L.dpg_set_real_path.argtypes = [vp, i32]
    L.dpg_cg_bytes_per_iteration.argtypes = [vp, i32, C.POINTER(i64)]
    L.dpg_timing_get.argtypes = [vp, C.POINTER(dpg_timing)]
    L.dpg_last_error.argtypes = [vp]
    L.dpg_last_error.restype = C.c_char_p
    L.dpg_destroy.argtypes = [vp]
    L.dpg_destroy.restype = None
    for name in ("dpg_setup_mesh", "dpg_element_batch", "dpg_assemble", "dpg_cg_solve", "dpg_estimate",
                 "dpg_estimate_noalloc",
                 "dpg_sizes", "dpg_trace_map", "dpg_element_dump", "dpg_csr_copy", "dpg_probe_peaks",
                 "dpg_update_elements", "dpg_timing_enable", "dpg_timing_get", "dpg_grad_eps",
                 "dpg_set_real_path", "dpg_cg_bytes_per_iteration", "dpg_element_layout", "dpg_tc_gemm", "dpg_set_graph", "dpg_autotune", "dpg_power",
                 "dpg_set_wait_limit", "dpg_set_factor_arith", "dpg_factor_check", "dpg_estimate_clamped", "dpg_mark_fraction",
                 "dpg_group_info", "dpg_set_bucketed", "dpg_factor_balance", "dpg_set_estimator_store"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def check(rc, h=None):
    if rc != DPG_OK:
        msg = lib().dpg_last_error(h)
        raise DPGError(rc, msg.decode() if msg else "")
    return rc


def ptr(t):
    """Data pointer of a tensor / numpy array (None -> NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(t.ctypes.data)


def stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)
