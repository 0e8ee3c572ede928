"""ctypes view of libchi0.so (include/chi0.h).  Loads the in-tree library and
fails loudly when it is missing; there is no fallback implementation."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchi0.so")

(CHI0_OK, CHI0_ERR_INVALID, CHI0_ERR_OOM, CHI0_ERR_CUDA, CHI0_ERR_TIMEOUT, CHI0_ERR_UNSUPPORTED,
 CHI0_ERR_SINGULAR) = range(7)
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "UNSUPPORTED", 6: "SINGULAR"}
CHI0_FP64, CHI0_SPLIT_BF16, CHI0_SPLIT_FP16 = 0, 1, 2
PRECISIONS = {"fp64": CHI0_FP64, "bf16": CHI0_SPLIT_BF16, "fp16": CHI0_SPLIT_FP16}


class Chi0PlanDesc(C.Structure):
    _fields_ = [
        ("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int),
        ("n_q", C.c_int),
        ("n_G", C.POINTER(C.c_int32)),
        ("gvec", C.POINTER(C.c_int32)),
        ("npw", C.c_int),
        ("gw", C.POINTER(C.c_int32)),
        ("n_freq", C.c_int),
        ("freq_re", C.POINTER(C.c_double)),
        ("freq_im", C.POINTER(C.c_double)),
        ("delta", C.c_double),
        ("precision", C.c_int),
        ("n_products", C.c_int),
        ("max_pairs", C.c_int64),
        ("chain_pairs", C.c_int),
        ("hermitian", C.c_int),
    ]


# (name, restype, argtypes) for every symbol declared in include/chi0.h
_VP, _I, _I64, _D = C.c_void_p, C.c_int, C.c_int64, C.c_double
SIGNATURES = [
    ("chi0_plan_create", _I, [C.POINTER(_VP), C.POINTER(Chi0PlanDesc)]),
    ("chi0_plan_destroy", _I, [_VP]),
    ("chi0_last_error", C.c_char_p, [_VP]),
    ("chi0_workspace_bytes", C.c_size_t, [_VP]),
    ("chi0_sync_status", _I, [_VP, _VP]),
    ("chi0_wfn_to_grid", _I, [_VP, _VP, _I, _VP, _VP]),
    ("chi0_pairs", _I, [_VP, _I, _VP, _VP, _I, _VP, _VP, _I, _VP, _VP]),
    ("chi0_accumulate", _I, [_VP, _I, _VP, _I, _I, _VP, _VP, _VP, _VP, _VP]),
    ("chi0_build", _I, [_VP, _I, _VP, _I, _VP, _VP, _VP, _I, _VP, _VP, _VP, _VP]),
    ("chi0_select_accelerated", _I, [_VP, _I, _I, _D, _D, _D, _D, _VP, _VP, _VP, _I]),
    ("chi0_select_quadrature", _I, [_VP, _I, _I, _D, _D, _D, _D, _I, _I, _I, _VP, _VP, _VP, _I]),
    ("chi0_select_adaptive", _I, [_VP, _I, _I, _VP, _D, _D, _D, _D, _I, _I, _VP, _VP, _VP, _I]),
    ("chi0_build_batched", _I, [_VP, _VP, _I, _VP, _VP, _VP, _I, _VP, _VP, _VP, _I, _VP]),
    ("chi0_backward", _I, [_VP, _I, _VP, _I, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("chi0_selftest_wait", _I, [_VP, _D, _VP]),
    ("chi0_coulomb", _I, [_VP, _I, _VP, _VP, _VP]),
    ("chi0_epsilon", _I, [_VP, _I, _VP, _VP, _I, _VP, _VP]),
    ("chi0_epsilon_inverse", _I, [_VP, _I, _VP, _VP]),
    ("chi0_eps_inf", _I, [_VP, _I, _VP, _VP, _VP]),
    ("chi0_gpp", _I, [_VP, _I, _VP, _I, _VP, _VP, _VP, _D, _VP, _VP, _VP]),
    ("chi0_sigma_coh", _I, [_VP, _I, _VP, _I, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("chi0_autotune", _I, [_VP, _I, _I, _VP, _VP]),
    ("chi0_get_tuning", _I, [_VP, _VP, _VP, _VP]),
    ("chi0_plan_hermitian", _I, [_VP, _VP]),
    ("chi0_profile_enable", _I, [_VP, _I]),
    ("chi0_profile_reset", _I, [_VP]),
    ("chi0_profile_read", _I, [_VP, _VP, _VP]),
    ("chi0_energy_substitution_estimate", _I, [_VP, _VP, _VP, _I, _I, _D, _D, _VP, _VP, _VP]),
    ("chi0_grid_energies", _I, [_VP, _I, _I, _D, _D, _VP]),
    ("chi0_peak_fma", _I, [_I, _I, _VP, _VP, _VP]),
    ("chi0_accumulate_fp64_noalloc", _I, [_I, _VP, _I, _I, _VP, _VP, _VP, _I, _VP, _VP, _D, _VP, _VP]),
]
KERNELS = ["wfn", "pair_planes", "pair_gather", "weights", "pack", "contract_tc", "contract_f64",
           "epsilon", "inv_panel", "inv_update"]

_lib = None


class Chi0Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"chi0 error {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib() -> C.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1601_06767_gb300.build` (there is no CPU fallback)")
        h = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def check(status: int, plan=None) -> None:
    if status != CHI0_OK:
        msg = lib().chi0_last_error(plan)
        raise Chi0Error(status, (msg or b"").decode(errors="replace"))
