"""Python binding of libfenc (the C ABI in include/fenc.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
PyTorch provides device memory (tensors are passed as raw pointers) and the
current CUDA stream.  Ciphertexts, plaintexts and keys are int64 tensors that
hold the uint64 residues bit for bit.

Importing the package does not need a GPU; creating a Context does, and the
library must have been built (paper_2606_16359_b300.build.build()).  There is no
fallback path: a missing library raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libfenc.so")

FE_OK, FE_EINVAL, FE_ENOMEM, FE_ELEVEL, FE_ESCALE, FE_EKEY, FE_ETIMEOUT, FE_ECUDA, FE_EENCODE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8

u32, u64, i32, sz, vp, dbl = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_size_t,
                              ctypes.c_void_p, ctypes.c_double)
cint = ctypes.c_int

# rotation-step value standing for the complex conjugation of the slots (Galois element 2N - 1)
FE_STEP_CONJ = -(1 << 31)


class FeParams(ctypes.Structure):
    _fields_ = [("logN", u32), ("n_q", u32), ("k", u32), ("qbits", u32), ("pbits", u32)]


class FeBootParams(ctypes.Structure):
    _fields_ = [("n_cts", u32), ("n_stc", u32), ("r", u32), ("top", u32), ("baby_ratio", u32),
                ("double_hoist", u32), ("form", u32)]


class FeLayout(ctypes.Structure):
    _fields_ = [(n, u32) for n in ("H", "W", "C", "BS", "S", "m", "M", "cpc", "groups", "n_ct")]

    def describe(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class FeCounters(ctypes.Structure):
    _fields_ = [(n, u64) for n in ("rot", "keyswitch", "ntt", "pmult", "cmult", "rescale", "launches")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class FePlanInfo(ctypes.Structure):
    _fields_ = [("pt_bytes", sz), ("in_bytes", sz), ("out_bytes", sz), ("workspace_bytes", sz),
                ("workspace_min_bytes", sz), ("n_in_ct", u32), ("n_out_ct", u32), ("n_pt", u32),
                ("n_inner_rot", u32), ("n_outer_rot", u32), ("bsgs_n1", u32), ("double_hoist", u32)]


P = ctypes.POINTER
# name: (restype, argtypes)
class FeRotationModel(ctypes.Structure):
    _fields_ = [("m", u32), ("M", u32), ("cpc", u32), ("alpha", dbl), ("eq3_inner", dbl), ("eq4_outer", dbl),
                ("eq5_total", dbl), ("s_bound_eq7", dbl), ("s_star_eq8", dbl), ("executed_inner", u64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class FeFragmentChoice(ctypes.Structure):
    _fields_ = [("S", u32), ("m", u32), ("M", u32), ("cpc", u32), ("n_admissible", u32), ("alpha", dbl),
                ("eq5", dbl), ("s_star", dbl)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class FeTokenLayout(ctypes.Structure):
    _fields_ = [("n_tok", u32), ("E", u32), ("S", u32), ("P", u32), ("F", u32), ("n_ct", u32)]


class FeServerConfig(ctypes.Structure):
    _fields_ = [("max_batch", u32), ("max_inflight", u32), ("hbm_budget_bytes", sz), ("hbm_reserve_bytes", sz)]


class FeOp(ctypes.Structure):
    _fields_ = [("kind", cint), ("plan", vp), ("pt_dev", vp), ("layout", FeLayout), ("a", dbl), ("b", dbl),
                ("c", dbl), ("in_scale", dbl), ("boot", vp)]


class FeServerStats(ctypes.Structure):
    _fields_ = [("submitted", u64), ("completed", u64), ("rejected", u64), ("groups", u64), ("max_group", u64),
                ("max_inflight", u64), ("peak_bytes", sz), ("budget_bytes", sz), ("p50_ms", dbl), ("p99_ms", dbl),
                ("mean_ms", dbl), ("wall_s", dbl)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


OP_LAYER, OP_SQUARE, OP_POOL, OP_POLY_ACT, OP_REFRESH = 0, 1, 2, 3, 4

SIGNATURES = {
    "fe_mlp_create": (cint, [u32, u32, u32, u64, P(vp)]),
    "fe_mlp_destroy": (None, [vp]),
    "fe_mlp_param_count": (sz, [vp]),
    "fe_mlp_get_params": (cint, [vp, P(ctypes.c_float)]),
    "fe_mlp_set_params": (cint, [vp, P(ctypes.c_float)]),
    "fe_mlp_get_scaling": (cint, [vp, P(ctypes.c_float), P(ctypes.c_float), P(ctypes.c_float)]),
    "fe_mlp_train": (cint, [vp, vp, vp, u32, u32, ctypes.c_float, ctypes.c_float, P(ctypes.c_float), vp]),
    "fe_mlp_predict": (cint, [vp, vp, u32, vp, vp]),
    "fe_evk_alias": (cint, [vp, vp, P(i32), u32, P(u32)]),
    "fe_he_layer_timing": (cint, [vp, vp, vp, vp, u32, vp, vp, vp, sz, vp]),
    "fe_plan_truncate": (cint, [vp, u32]),
    "fe_device_status": (cint, [vp, P(u32), cint]),
    "fe_ctx_set_mac_wait": (cint, [vp, u64, i32]),
    "fe_plan_set_mac_ways": (cint, [vp, u32]),
    "fe_plan_set_lift_fusion": (cint, [vp, cint]),
    "fe_plan_set_hoisting": (cint, [vp, cint]),
    "fe_server_create": (cint, [P(FeServerConfig), P(vp)]),
    "fe_server_add_model": (cint, [vp, vp, vp, P(FeOp), u32, u32, u32, P(u32)]),
    "fe_server_model_io": (cint, [vp, u32, P(u32), P(u32), P(sz), P(sz)]),
    "fe_server_submit": (cint, [vp, u32, vp, vp, P(u64)]),
    "fe_server_pause": (cint, [vp, cint]),
    "fe_server_wait": (cint, [vp, u64, u32, P(cint), P(dbl)]),
    "fe_server_stats": (cint, [vp, P(FeServerStats)]),
    "fe_server_destroy": (None, [vp]),
    "fe_rotation_model": (cint, [u32, u32, u32, u32, u32, u32, u32, u32, u32, cint, P(FeRotationModel)]),
    "fe_choose_fragment": (cint, [u32, u32, u32, u32, u32, u32, u32, cint, u32, P(FeFragmentChoice)]),
    "fe_ctx_create": (cint, [P(FeParams), P(vp)]),
    "fe_ctx_destroy": (None, [vp]),
    "fe_ctx_moduli": (cint, [vp, P(u64)]),
    "fe_ctx_set_generator": (cint, [vp, cint, P(u32)]),
    "fe_evk_upload": (cint, [vp, vp, sz, P(i32), u32, cint, vp, sz, vp, P(vp)]),
    "fe_ctx_set_ntt_radix": (cint, [vp, cint]),
    "fe_ctx_set_ntt_q36": (cint, [vp, cint]),
    "fe_ctx_set_ntt_path": (cint, [vp, cint]),
    "fe_ctx_set_ntt_forward": (cint, [vp, cint]),
    "fe_get_counters": (cint, [vp, P(FeCounters)]),
    "fe_counters_reset": (cint, [vp]),
    "fe_last_error": (ctypes.c_char_p, []),
    "fe_sk_gen": (cint, [vp, u64, vp, vp]),
    "fe_evk_bytes": (sz, [vp, u32, cint]),
    "fe_evk_gen": (cint, [vp, vp, u64, P(i32), u32, cint, vp, sz, vp, P(vp)]),
    "fe_evk_destroy": (None, [vp]),
    "fe_layout_make": (cint, [vp, P(FeLayout)]),
    "fe_fragment_pack": (cint, [vp, P(FeLayout), vp, vp, vp]),
    "fe_fragment_unpack": (cint, [vp, P(FeLayout), vp, vp, vp]),
    "fe_encode": (cint, [vp, vp, u32, u32, dbl, vp, vp]),
    "fe_encode_encrypt": (cint, [vp, vp, vp, u32, u32, dbl, u64, u64, vp, vp]),
    "fe_decrypt_decode": (cint, [vp, vp, vp, u32, u32, dbl, vp, vp]),
    "fe_ntt": (cint, [vp, vp, u32, u32, u32, cint, vp]),
    "fe_probe_butterflies": (cint, [vp, u32, u32, vp, P(u64), vp]),
    "fe_rotate": (cint, [vp, vp, vp, u32, u32, i32, vp, vp]),
    "fe_rotate_many": (cint, [vp, vp, vp, u32, u32, P(i32), u32, vp, vp]),
    "fe_rescale": (cint, [vp, vp, u32, u32, vp, vp]),
    "fe_rescale_noalloc": (cint, [vp, vp, u32, u32, vp, vp]),
    "fe_pmult": (cint, [vp, vp, vp, u32, u32, vp, vp]),
    "fe_add": (cint, [vp, vp, vp, u32, u32, vp, vp]),
    "fe_plan_conv": (cint, [vp, P(FeLayout), u32, u32, u32, cint, u32, u32, u32, P(FeLayout), P(vp)]),
    "fe_plan_fc": (cint, [vp, u32, u32, u32, P(i32), u32, u32, u32, P(vp)]),
    "fe_plan_destroy": (None, [vp]),
    "fe_plan_fc_layout": (cint, [vp, P(FeLayout), u32, u32, P(vp)]),
    "fe_plan_fc_next": (cint, [vp, vp, u32, u32, P(vp)]),
    "fe_plan_repack": (cint, [vp, P(FeLayout), P(FeLayout), u32, P(vp)]),
    "fe_token_layout_make": (cint, [vp, P(FeTokenLayout)]),
    "fe_token_pack": (cint, [vp, P(FeTokenLayout), vp, vp, vp]),
    "fe_token_unpack": (cint, [vp, P(FeTokenLayout), vp, vp, vp]),
    "fe_plan_token_linear": (cint, [vp, P(FeTokenLayout), u32, u32, P(FeTokenLayout), P(vp)]),
    "fe_choose_token_fragment": (cint, [u32, u32, dbl, u32, P(u32), P(dbl), P(dbl)]),
    "fe_attention_rotation_steps": (cint, [vp, P(FeTokenLayout), P(i32), u32, P(u32)]),
    "fe_he_attention_scores": (cint, [vp, vp, P(FeTokenLayout), vp, vp, u32, dbl, dbl, vp, P(dbl), vp]),
    "fe_he_attention_apply": (cint, [vp, vp, P(FeTokenLayout), vp, u32, dbl, vp, u32, dbl, vp, P(u32), P(dbl), vp]),
    "fe_he_repack": (cint, [vp, vp, vp, vp, vp, vp, vp, sz, cint, vp]),
    "fe_fc_unpack": (cint, [vp, vp, vp, vp, vp]),
    "fe_weight_scale": (cint, [vp, u32, dbl, dbl, dbl, P(dbl)]),
    "fe_plan_out_scale": (cint, [vp, dbl, P(dbl)]),
    "fe_poly_act_workspace_bytes": (sz, [vp, u32, u32]),
    "fe_poly_act_scale": (cint, [vp, u32, dbl, dbl, P(dbl)]),
    "fe_he_poly_act": (cint, [vp, vp, dbl, dbl, dbl, vp, u32, u32, dbl, vp, P(dbl), vp, sz, vp]),
    "fe_compress_masked_workspace_bytes": (sz, [vp, u32, u32]),
    "fe_compress_masked": (cint, [vp, vp, P(FeLayout), u32, dbl, vp, u32, u32, dbl, vp, P(dbl), vp, sz, vp]),
    "fe_plan_query": (cint, [vp, P(FePlanInfo)]),
    "fe_plan_rotation_steps": (cint, [vp, P(i32), u32, P(u32)]),
    "fe_plan_load_weights": (cint, [vp, vp, vp, dbl, dbl, vp, vp]),
    "fe_he_conv": (cint, [vp, vp, vp, vp, vp, vp, vp, sz, cint, vp]),
    "fe_plan_workspace_bytes": (sz, [vp, u32, cint]),
    "fe_he_layer_batch": (cint, [vp, vp, vp, vp, vp, vp, u32, vp, sz, cint, vp]),
    "fe_he_fc": (cint, [vp, vp, vp, vp, vp, vp, vp, sz, cint, vp]),
    "fe_square_workspace_bytes": (sz, [vp, u32, u32]),
    "fe_he_square": (cint, [vp, vp, vp, u32, u32, vp, vp, sz, vp]),
    "fe_he_avgpool": (cint, [vp, P(FeLayout), vp, u32, vp, P(FeLayout), vp]),
    "fe_compress_workspace_bytes": (sz, [vp, u32, u32]),
    "fe_compress": (cint, [vp, vp, P(FeLayout), u32, vp, u32, u32, vp, vp, sz, vp]),
    "fe_graph_capture": (cint, [vp, vp, P(vp), P(vp), P(vp), P(vp), u32, vp, sz, vp, P(vp)]),
    "fe_graph_capture_batch": (cint, [vp, vp, P(vp), P(vp), P(vp), P(vp), u32, u32, vp, sz, vp, P(vp)]),
    "fe_graph_workspace_bytes": (sz, [P(vp), u32, u32]),
    "fe_graph_workspace_bytes_chunked": (sz, [P(vp), u32, u32, u32]),
    "fe_graph_capture_chunked": (cint, [vp, vp, P(vp), P(vp), P(vp), P(vp), u32, u32, u32, vp, sz, vp, P(vp)]),
    "fe_graph_launch": (cint, [vp, vp]),
    "fe_graph_io": (cint, [vp, P(u32), P(sz), P(u32), P(sz)]),
    "fe_graph_launch_host": (cint, [vp, P(vp), P(vp), vp]),
    "fe_graph_set_host_output_level": (cint, [vp, u32]),
    "fe_graph_destroy": (None, [vp]),
    "fe_sk_gen_sparse": (cint, [vp, u64, u32, vp, vp]),
    "fe_conjugate": (cint, [vp, vp, vp, u32, u32, vp, vp]),
    "fe_mod_raise": (cint, [vp, vp, u32, u32, vp, vp]),
    "fe_mod_drop": (cint, [vp, vp, u32, u32, u32, vp, vp]),
    "fe_plan_lintrans": (cint, [vp, u32, u32, u32, P(u32), P(u32), P(i32), u32, u32, P(vp)]),
    "fe_plan_lintrans_load": (cint, [vp, vp, vp, dbl, vp, vp]),
    "fe_he_lintrans": (cint, [vp, vp, vp, vp, vp, vp, u32, vp, sz, vp]),
    "fe_boot_create": (cint, [vp, P(FeBootParams), dbl, vp, P(vp)]),
    "fe_boot_rotation_steps": (cint, [vp, P(i32), u32, P(u32)]),
    "fe_boot_output": (cint, [vp, P(u32), P(dbl)]),
    "fe_boot_workspace_bytes": (sz, [vp, u32]),
    "fe_he_bootstrap": (cint, [vp, vp, vp, vp, u32, vp, vp, sz, vp]),
    "fe_boot_graph_capture": (cint, [vp, vp, vp, vp, u32, vp, vp, sz, vp, P(vp)]),
    "fe_boot_destroy": (None, [vp]),
    "fe_boot_prepare_workspace_bytes": (sz, [vp, u32]),
    "fe_swk_gen": (cint, [vp, vp, vp, u64, u32, vp, sz, vp]),
    "fe_key_switch": (cint, [vp, vp, vp, u32, u32, vp, vp]),
    "fe_boot_encapsulate": (cint, [vp, vp, vp, vp, u64, vp, sz, vp]),
    "fe_boot_prepare": (cint, [vp, vp, vp, u32, u32, dbl, vp, vp, sz, vp]),
    "fe_profile_begin": (cint, [vp, ctypes.c_char_p]),
    "fe_profile_end": (cint, [vp, P(dbl), P(u64), P(dbl)]),
}

_lib = None


def load():
    """Load libfenc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfenc.so is not built ({LIB_PATH}); run paper_2606_16359_b300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class FencError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def check(rc):
    if rc != FE_OK:
        raise FencError(rc, load().fe_last_error().decode())
    return rc


def _torch():
    import torch
    return torch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


class Evk:
    """Switching keys held in a torch buffer, with the library handle."""

    def __init__(self, ctx, handle, buf, steps, relin):
        self.ctx, self.handle, self.buf, self.steps, self.relin = ctx, handle, buf, list(steps), relin

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fe_evk_destroy(self.handle)
            self.handle = None


class Plan:
    def __init__(self, ctx, handle, out_layout=None):
        self.ctx, self.handle, self.out_layout = ctx, handle, out_layout
        self.refresh()

    def refresh(self):
        handle = self.handle
        info = FePlanInfo()
        check(load().fe_plan_query(handle, ctypes.byref(info)))
        self.info = info
        n = u32()
        check(load().fe_plan_rotation_steps(handle, None, 0, ctypes.byref(n)))
        arr = (i32 * max(1, n.value))()
        check(load().fe_plan_rotation_steps(handle, arr, n.value, ctypes.byref(n)))
        self.steps = [arr[i] for i in range(n.value)]

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fe_plan_destroy(self.handle)
            self.handle = None


class Boot:
    """A ciphertext refresh built by Context.boot_create (fe_boot_create)."""

    def __init__(self, ctx, handle, scale_in):
        self.ctx, self.handle, self.scale_in = ctx, handle, scale_in
        n = u32()
        check(load().fe_boot_rotation_steps(handle, None, 0, ctypes.byref(n)))
        arr = (i32 * max(1, n.value))()
        check(load().fe_boot_rotation_steps(handle, arr, n.value, ctypes.byref(n)))
        self.steps = [arr[i] for i in range(n.value)]
        lv, sc = u32(), dbl()
        check(load().fe_boot_output(handle, ctypes.byref(lv), ctypes.byref(sc)))
        self.out_level, self.out_scale = lv.value, sc.value

    def workspace_bytes(self, n_ct=1):
        return int(load().fe_boot_workspace_bytes(self.handle, n_ct))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fe_boot_destroy(self.handle)
            self.handle = None


def _hoisting(v):
    """fe_plan_set_hoisting's value: False / 0, True / 1, 2 or "fused"."""
    if v == "fused":
        return 2
    if v is True:
        return 1
    if v in (0, 1, 2):
        return int(v)
    raise ValueError(f"hoisting must be False, True, 2 or 'fused', not {v!r}")


class Graph:
    def __init__(self, handle, keep):
        self.handle, self._keep = handle, keep

    def launch(self):
        check(load().fe_graph_launch(self.handle, _stream()))

    def io(self):
        """(input byte sizes, output byte sizes) of the graph's host-visible ends."""
        ni, no = u32(0), u32(0)
        check(load().fe_graph_io(self.handle, ctypes.byref(ni), None, ctypes.byref(no), None))
        ib, ob = (sz * max(1, ni.value))(), (sz * max(1, no.value))()
        check(load().fe_graph_io(self.handle, ctypes.byref(ni), ib, ctypes.byref(no), ob))
        return list(ib)[:ni.value], list(ob)[:no.value]

    def set_host_output_level(self, level=None):
        """Final outputs reach the host at `level` (exact modulus drop); None: their own level."""
        check(load().fe_graph_set_host_output_level(self.handle, 0xFFFFFFFF if level is None else int(level)))

    def launch_host(self, in_host, out_host):
        """One step through host memory (copies in, replay, copies out) on the current stream.
        in_host / out_host: host tensors (pinned for asynchronous copies) of io()'s sizes."""
        ib, ob = self.io()
        assert len(in_host) == len(ib) and len(out_host) == len(ob)
        for t, b in zip(list(in_host) + list(out_host), ib + ob):
            assert not t.is_cuda and t.numel() * t.element_size() == b
        ins = (vp * max(1, len(ib)))(*[t.data_ptr() for t in in_host])
        outs = (vp * max(1, len(ob)))(*[t.data_ptr() for t in out_host])
        check(load().fe_graph_launch_host(self.handle, ins, outs, _stream()))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fe_graph_destroy(self.handle)
            self.handle = None


class Context:
    """An RNS-CKKS parameter set on the current CUDA device."""

    def __init__(self, logN, n_q, k, qbits, pbits=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        lib = load()
        self.params = FeParams(logN, n_q, k, qbits, qbits if pbits is None else pbits)
        h = vp()
        check(lib.fe_ctx_create(ctypes.byref(self.params), ctypes.byref(h)))
        self.handle = h
        self.logN, self.N, self.L, self.k = logN, 1 << logN, n_q - 1, k
        self.n_mod = n_q + k
        arr = (u64 * self.n_mod)()
        check(lib.fe_ctx_moduli(h, arr))
        self.moduli = [int(arr[i]) for i in range(self.n_mod)]

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fe_ctx_destroy(self.handle)
            self.handle = None

    # -- helpers --------------------------------------------------------------
    def ct_words(self, level):
        return 2 * (level + 1) * self.N

    def empty_ct(self, n, level):
        return _torch().empty((n, 2, level + 1, self.N), dtype=_torch().int64, device="cuda")

    def counters(self):
        c = FeCounters()
        check(load().fe_get_counters(self.handle, ctypes.byref(c)))
        return c.as_dict()

    def reset_counters(self):
        check(load().fe_counters_reset(self.handle))

    # -- keys -------------------------------------------------------------------
    def sk_gen(self, seed):
        sk = _torch().empty((self.n_mod, self.N), dtype=_torch().int64, device="cuda")
        check(load().fe_sk_gen(self.handle, seed, _ptr(sk), _stream()))
        return sk

    def sk_gen_sparse(self, seed, h):
        """Sparse ternary secret of Hamming weight h (fe_sk_gen_sparse)."""
        sk = _torch().empty((self.n_mod, self.N), dtype=_torch().int64, device="cuda")
        check(load().fe_sk_gen_sparse(self.handle, seed, h, _ptr(sk), _stream()))
        return sk

    def evk_gen(self, sk, seed, steps, relin=False):
        steps = sorted({int(s) for s in steps})
        nbytes = load().fe_evk_bytes(self.handle, len(steps), 1 if relin else 0)
        buf = _torch().empty(max(8, nbytes) // 8, dtype=_torch().int64, device="cuda")
        arr = (i32 * max(1, len(steps)))(*steps)
        h = vp()
        check(load().fe_evk_gen(self.handle, _ptr(sk), seed, arr, len(steps), 1 if relin else 0, _ptr(buf),
                                nbytes, _stream(), ctypes.byref(h)))
        return Evk(self, h, buf, steps, relin)

    def evk_upload(self, host, steps, relin=False):
        """Index switching keys produced elsewhere (host: an int64 CPU tensor in
        evk_gen's layout for `steps` in the given order), on this device."""
        torch = _torch()
        steps = [int(s) for s in steps]
        nbytes = load().fe_evk_bytes(self.handle, len(steps), 1 if relin else 0)
        host = host.contiguous()
        buf = torch.empty(max(8, nbytes) // 8, dtype=torch.int64, device="cuda")
        arr = (i32 * max(1, len(steps)))(*steps)
        h = vp()
        check(load().fe_evk_upload(self.handle, ctypes.c_void_p(host.data_ptr()), host.numel() * 8, arr, len(steps),
                                   1 if relin else 0, _ptr(buf), nbytes, _stream(), ctypes.byref(h)))
        return Evk(self, h, buf, steps, relin)

    # -- client side --------------------------------------------------------------
    def layout(self, H, W, C, BS, S, m=0):
        lay = FeLayout(H, W, C, BS, S, m, 0, 0, 0, 0)
        check(load().fe_layout_make(self.handle, ctypes.byref(lay)))
        return lay

    def pack(self, lay, x):
        torch = _torch()
        x = torch.as_tensor(x, dtype=torch.float64).cuda().contiguous()
        slots = torch.empty((lay.n_ct, self.N // 2), dtype=torch.float64, device="cuda")
        check(load().fe_fragment_pack(self.handle, ctypes.byref(lay), _ptr(x), _ptr(slots), _stream()))
        return slots

    def unpack(self, lay, slots):
        torch = _torch()
        y = torch.empty((lay.BS, lay.C, lay.H, lay.W), dtype=torch.float64, device="cuda")
        check(load().fe_fragment_unpack(self.handle, ctypes.byref(lay), _ptr(slots.contiguous()), _ptr(y), _stream()))
        return y

    def encode(self, slots, level, scale):
        torch = _torch()
        slots = torch.as_tensor(slots, dtype=torch.float64).cuda().contiguous()
        n = slots.shape[0]
        pt = torch.empty((n, level + 1, self.N), dtype=torch.int64, device="cuda")
        check(load().fe_encode(self.handle, _ptr(slots), n, level, scale, _ptr(pt), _stream()))
        return pt

    def encrypt(self, sk, slots, level, scale, seed, ct_id0=0):
        torch = _torch()
        slots = torch.as_tensor(slots, dtype=torch.float64).cuda().contiguous()
        n = slots.shape[0]
        ct = self.empty_ct(n, level)
        check(load().fe_encode_encrypt(self.handle, _ptr(sk), _ptr(slots), n, level, scale, seed, ct_id0,
                                       _ptr(ct), _stream()))
        return ct

    def decrypt(self, sk, ct, level, scale):
        torch = _torch()
        n = ct.shape[0]
        out = torch.empty((n, self.N // 2), dtype=torch.float64, device="cuda")
        check(load().fe_decrypt_decode(self.handle, _ptr(sk), _ptr(ct), n, level, scale, _ptr(out), _stream()))
        return out

    def set_generator(self, kind, key_material=None):
        """Generator of every sampler: "splitmix64" (default) or "chacha20" keyed by
        (seed, key_material: six 32-bit words) (see fe_ctx_set_generator)."""
        code = {"splitmix64": 0, "chacha20": 1}[kind]
        arr = (u32 * 6)(*[int(v) & 0xFFFFFFFF for v in (key_material if key_material is not None else [0] * 6)])
        check(load().fe_ctx_set_generator(self.handle, code, arr))

    def set_ntt_radix(self, radix):
        check(load().fe_ctx_set_ntt_radix(self.handle, radix))

    def set_ntt_q36(self, enable):
        check(load().fe_ctx_set_ntt_q36(self.handle, int(enable)))

    def set_ntt_forward(self, flags):
        """bit 0: reduce every forward stage to [0, 4q); bit 1: 36-bit Shoup product forward."""
        check(load().fe_ctx_set_ntt_forward(self.handle, int(flags)))

    def set_ntt_path(self, path):
        """0: two passes (first and last rounds on global memory); 1: two passes
        staged through shared memory; 2: one pass on clusters of 8 CTAs (N = 2^16)."""
        check(load().fe_ctx_set_ntt_path(self.handle, int(path)))

    # -- primitives ------------------------------------------------------------------
    def ntt(self, data, first_mod=0, inverse=False):
        n_poly, n_limbs = data.shape[0], data.shape[1]
        check(load().fe_ntt(self.handle, _ptr(data), n_poly, n_limbs, first_mod, 1 if inverse else 0, _stream()))
        return data

    def probe_butterflies(self, out, blocks, iters):
        """Launch the butterfly-throughput probe; returns the butterflies executed."""
        n = ctypes.c_uint64(0)
        check(load().fe_probe_butterflies(self.handle, blocks, iters, _ptr(out), ctypes.byref(n), _stream()))
        return n.value

    def rotate(self, evk, ct, level, r):
        out = self.empty_ct(ct.shape[0], level)
        check(load().fe_rotate(self.handle, evk.handle, _ptr(ct), ct.shape[0], level, r, _ptr(out), _stream()))
        return out

    def rotate_many(self, evk, ct, level, steps):
        """Hoisted rotations: returns [len(steps), n_ct, 2, level + 1, N], entry j = rotate(ct, steps[j])."""
        n, k = ct.shape[0], len(steps)
        out = _torch().empty((k, n, 2, level + 1, self.N), dtype=_torch().int64, device="cuda")
        arr = (i32 * max(1, k))(*steps)
        check(load().fe_rotate_many(self.handle, evk.handle, _ptr(ct), n, level, arr, k, _ptr(out), _stream()))
        return out

    def conjugate(self, evk, ct, level):
        out = self.empty_ct(ct.shape[0], level)
        check(load().fe_conjugate(self.handle, evk.handle, _ptr(ct), ct.shape[0], level, _ptr(out), _stream()))
        return out

    def mod_drop(self, ct, level, to_level):
        """The ciphertexts modulo Q_to_level (exact, same scale; fe_mod_drop)."""
        out = self.empty_ct(ct.shape[0], to_level)
        check(load().fe_mod_drop(self.handle, _ptr(ct), ct.shape[0], level, to_level, _ptr(out), _stream()))
        return out

    def mod_raise(self, ct, top):
        out = self.empty_ct(ct.shape[0], top)
        check(load().fe_mod_raise(self.handle, _ptr(ct), ct.shape[0], top, _ptr(out), _stream()))
        return out

    def plan_lintrans(self, diags, n_in, n_out, level, n1=0):
        """Plaintext-matrix product over the diagonals [(out, in, offset), ...]
        (fe_plan_lintrans); the values are loaded with lintrans_load in this order."""
        d = np.asarray(diags, dtype=np.int64).reshape(-1, 3)
        o = np.ascontiguousarray(d[:, 0], dtype=np.uint32)
        i = np.ascontiguousarray(d[:, 1], dtype=np.uint32)
        r = np.ascontiguousarray(d[:, 2], dtype=np.int32)
        h = vp()
        check(load().fe_plan_lintrans(self.handle, n_in, n_out, len(d), o.ctypes.data_as(P(u32)),
                                      i.ctypes.data_as(P(u32)), r.ctypes.data_as(P_i32), n1, level, ctypes.byref(h)))
        p = Plan(self, h)
        p.level = level
        return p

    def lintrans_load(self, plan, values, w_scale=None):
        torch = _torch()
        v = np.ascontiguousarray(values, dtype=np.float64)
        w_scale = float(self.moduli[plan.level]) if w_scale is None else w_scale
        pt = torch.empty(max(8, plan.info.pt_bytes) // 8, dtype=torch.int64, device="cuda")
        check(load().fe_plan_lintrans_load(self.handle, plan.handle, v.ctypes.data_as(vp), w_scale, _ptr(pt),
                                           _stream()))
        return pt

    def he_lintrans(self, evk, plan, pt, ct, n_req=1, ws=None, out=None):
        ws = self.workspace(self.workspace_bytes(plan, n_req)) if ws is None else ws
        out = self.empty_ct(n_req * plan.info.n_out_ct, plan.level - 1) if out is None else out
        self._check_layer_buffers(plan, pt, ct, out, n_req)
        check(load().fe_he_lintrans(self.handle, evk.handle, plan.handle, _ptr(pt), _ptr(ct), _ptr(out), n_req,
                                    _ptr(ws), ws.numel() * 8, _stream()))
        return out

    def boot_create(self, scale_in, n_cts=3, n_stc=3, r=6, top=0, baby_ratio=4, double_hoist=True, form="complex"):
        """A ciphertext refresh (fe_boot_create) for level-0 inputs at scale_in
        (form: "real" or "complex", see fe_boot_params)."""
        prm = FeBootParams(n_cts, n_stc, r, top, baby_ratio, 1 if double_hoist else 0,
                           {"real": 0, "complex": 1}[form])
        h = vp()
        check(load().fe_boot_create(self.handle, ctypes.byref(prm), scale_in, _stream(), ctypes.byref(h)))
        return Boot(self, h, scale_in)

    def swk_gen(self, sk_src, sk_dst, seed, obj):
        """Switching key sk_src -> sk_dst (fe_swk_gen), one rotation key's layout."""
        nbytes = load().fe_evk_bytes(self.handle, 1, 0)
        key = _torch().empty(nbytes // 8, dtype=_torch().int64, device="cuda")
        check(load().fe_swk_gen(self.handle, _ptr(sk_src), _ptr(sk_dst), seed, obj, _ptr(key), nbytes, _stream()))
        return key

    def key_switch(self, key, ct, level):
        out = self.empty_ct(ct.shape[0], level)
        check(load().fe_key_switch(self.handle, _ptr(key), _ptr(ct), ct.shape[0], level, _ptr(out), _stream()))
        return out

    def boot_encapsulate(self, boot, sk_dense, sk_sparse, seed):
        """Let the refresh run under a dense secret (fe_boot_encapsulate); the two
        keys are kept on the Boot object."""
        nbytes = 2 * load().fe_evk_bytes(self.handle, 1, 0)
        keys = _torch().empty(nbytes // 8, dtype=_torch().int64, device="cuda")
        check(load().fe_boot_encapsulate(self.handle, boot.handle, _ptr(sk_dense), _ptr(sk_sparse), seed, _ptr(keys),
                                         nbytes, _stream()))
        boot.encaps_keys = keys
        return keys

    def boot_prepare(self, boot, ct, level, in_scale):
        """Ciphertexts at `level` (scale in_scale) to level 0 at boot.scale_in (fe_boot_prepare)."""
        n = ct.shape[0]
        ws = self.workspace(load().fe_boot_prepare_workspace_bytes(self.handle, n))
        out = self.empty_ct(n, 0)
        check(load().fe_boot_prepare(self.handle, boot.handle, _ptr(ct), n, level, float(in_scale), _ptr(out),
                                     _ptr(ws), ws.numel() * 8, _stream()))
        return out

    def bootstrap(self, evk, boot, ct, ws=None, out=None):
        """Refresh level-0 ciphertexts; returns them at boot.out_level (scale boot.out_scale)."""
        n = ct.shape[0]
        if ct.numel() != n * self.ct_words(0):
            raise ValueError("the refresh takes level-0 ciphertexts")
        ws = self.workspace(boot.workspace_bytes(n)) if ws is None else ws
        out = self.empty_ct(n, boot.out_level) if out is None else out
        if out.numel() != n * self.ct_words(boot.out_level):
            raise ValueError("output buffer does not match the refresh's output level")
        check(load().fe_he_bootstrap(self.handle, evk.handle, boot.handle, _ptr(ct), n, _ptr(out), _ptr(ws),
                                     ws.numel() * 8, _stream()))
        return out

    def boot_graph_capture(self, evk, boot, ct, out, ws):
        """One CUDA graph of the refresh of ct (level 0) into out, on the current
        (non-default) stream; replays give bootstrap()'s residues on the same buffers."""
        n = ct.shape[0]
        if ct.numel() != n * self.ct_words(0) or out.numel() != n * self.ct_words(boot.out_level):
            raise ValueError("the refresh takes level-0 ciphertexts into boot.out_level outputs")
        h = ctypes.c_void_p()
        check(load().fe_boot_graph_capture(self.handle, evk.handle, boot.handle, _ptr(ct), n, _ptr(out), _ptr(ws),
                                           ws.numel() * 8, _stream(), ctypes.byref(h)))
        return Graph(h, (evk, boot, ct, out, ws))

    def rescale(self, ct, level):
        out = self.empty_ct(ct.shape[0], level - 1)
        check(load().fe_rescale(self.handle, _ptr(ct), ct.shape[0], level, _ptr(out), _stream()))
        return out

    def pmult(self, ct, pt, level):
        out = self.empty_ct(ct.shape[0], level)
        check(load().fe_pmult(self.handle, _ptr(ct), _ptr(pt), ct.shape[0], level, _ptr(out), _stream()))
        return out

    def add(self, a, b, level):
        out = self.empty_ct(a.shape[0], level)
        check(load().fe_add(self.handle, _ptr(a), _ptr(b), a.shape[0], level, _ptr(out), _stream()))
        return out

    # -- layers -------------------------------------------------------------------------
    def plan_conv(self, lay, Cout, K, stride=1, depthwise=False, in_period=0, level=None, bsgs_n1=0,
                  double_hoist=False):
        level = self.L if level is None else level
        out_lay = FeLayout()
        h = vp()
        check(load().fe_plan_conv(self.handle, ctypes.byref(lay), Cout, K, stride, 1 if depthwise else 0,
                                  in_period, level, bsgs_n1, ctypes.byref(out_lay), ctypes.byref(h)))
        if double_hoist:
            check(load().fe_plan_set_hoisting(h, _hoisting(double_hoist)))
        p = Plan(self, h, out_lay)
        p.level, p.in_layout = level, lay
        return p

    def plan_fc(self, n_in_ct, P, BS, feat, F_in, F_out, level):
        feat = np.ascontiguousarray(feat, dtype=np.int32)
        h = vp()
        check(load().fe_plan_fc(self.handle, n_in_ct, P, BS, feat.ctypes.data_as(P_i32), F_in, F_out, level,
                                ctypes.byref(h)))
        p = Plan(self, h)
        p.level = level
        return p

    def load_weights(self, plan, W, w_scale, wmul=1.0):
        torch = _torch()
        W = np.ascontiguousarray(W, dtype=np.float64)
        pt = torch.empty(max(8, plan.info.pt_bytes) // 8, dtype=torch.int64, device="cuda")
        check(load().fe_plan_load_weights(self.handle, plan.handle, W.ctypes.data_as(vp), wmul, w_scale, _ptr(pt),
                                          _stream()))
        return pt

    def workspace(self, nbytes):
        return _torch().empty(max(8, (nbytes + 7) // 8), dtype=_torch().int64, device="cuda")

    def _check_layer_buffers(self, plan, pt, ct, out, n_req=1):
        """The device buffers a planned layer reads and writes must have the sizes its
        plan implies (the C ABI takes raw pointers and cannot see their extents)."""
        i = plan.info
        if ct.numel() != n_req * i.n_in_ct * self.ct_words(plan.level):
            raise ValueError(f"input holds {ct.numel()} words, the plan reads "
                             f"{n_req * i.n_in_ct} ciphertexts at level {plan.level}")
        if out.numel() != n_req * i.n_out_ct * self.ct_words(plan.level - 1):
            raise ValueError("output buffer does not match the plan")
        if pt.numel() * pt.element_size() < i.pt_bytes:
            raise ValueError("plaintext buffer smaller than the plan's pt_bytes")

    def he_conv(self, evk, plan, pt, ct, mode=1, ws=None, out=None):
        ws = self.workspace(plan.info.workspace_bytes) if ws is None else ws
        out = self.empty_ct(plan.info.n_out_ct, plan.level - 1) if out is None else out
        self._check_layer_buffers(plan, pt, ct, out)
        check(load().fe_he_conv(self.handle, evk.handle, plan.handle, _ptr(pt), _ptr(ct), _ptr(out), _ptr(ws),
                                ws.numel() * 8, mode, _stream()))
        return out

    def workspace_bytes(self, plan, n_req=1, minimum=False):
        return int(load().fe_plan_workspace_bytes(plan.handle, n_req, 1 if minimum else 0))

    def evk_alias(self, evk, steps):
        """Timing only: map keyless steps to generated keys (see fe_evk_alias)."""
        arr = (i32 * max(1, len(steps)))(*steps)
        n = u32(0)
        check(load().fe_evk_alias(self.handle, evk.handle, arr, len(steps), ctypes.byref(n)))
        return n.value

    def device_status(self, reset=False):
        """Synchronise and read the device status word (0: no bounded wait expired)."""
        v = u32(0)
        check(load().fe_device_status(self.handle, ctypes.byref(v), 1 if reset else 0))
        return v.value

    def set_mac_wait(self, limit_ns=2_000_000_000, unfed_term=-1):
        check(load().fe_ctx_set_mac_wait(self.handle, int(limit_ns), int(unfed_term)))

    def plan_set_hoisting(self, plan, double):
        """Hoisting of the plan's rotations (set before load_weights): False / 0
        single, True / 1 double, 2 or "fused" double with ModDown and rescale in
        one step when the plan has no outer rotation."""
        check(load().fe_plan_set_hoisting(plan.handle, _hoisting(double)))
        plan.refresh()
        return plan

    def plan_set_mac_ways(self, plan, ways):
        check(load().fe_plan_set_mac_ways(plan.handle, ways))
        plan.mac_ways = ways

    def plan_set_lift_fusion(self, plan, enable):
        """Depthwise double-hoisted plans: the MAC forms the rotated copies (1) or a lift pass writes them (0)."""
        check(load().fe_plan_set_lift_fusion(plan.handle, int(enable)))
        return plan

    def plan_truncate(self, plan, max_out_ct):
        check(load().fe_plan_truncate(plan.handle, max_out_ct))
        plan.refresh()
        return plan

    def he_layer_timing(self, evk, plan, pt_pool, n_pool, ct, out, ws):
        check(load().fe_he_layer_timing(self.handle, evk.handle, plan.handle, _ptr(pt_pool), n_pool, _ptr(ct),
                                        _ptr(out), _ptr(ws), ws.numel() * ws.element_size(), _stream()))
        return out

    def he_layer_batch(self, evk, plan, pt, ct, n_req, mode=1, ws=None, out=None):
        """One conv / FC layer for n_req requests laid out [n_req][n_in_ct] (ct: a
        tensor [n_req * n_in_ct, 2, level+1, N]); returns [n_req * n_out_ct, ...]."""
        info = plan.info
        lv = plan.level
        if out is None:
            out = self.empty_ct(n_req * info.n_out_ct, lv - 1)
        if ws is None:
            ws = self.workspace(self.workspace_bytes(plan, n_req))
        self._check_layer_buffers(plan, pt, ct, out, n_req)
        check(load().fe_he_layer_batch(self.handle, evk.handle, plan.handle, _ptr(pt), _ptr(ct), _ptr(out), n_req,
                                       _ptr(ws), ws.numel() * ws.element_size(), mode, _stream()))
        return out

    def he_fc(self, evk, plan, pt, ct, mode=1, ws=None, out=None):
        ws = self.workspace(plan.info.workspace_bytes) if ws is None else ws
        out = self.empty_ct(plan.info.n_out_ct, plan.level - 1) if out is None else out
        self._check_layer_buffers(plan, pt, ct, out)
        check(load().fe_he_fc(self.handle, evk.handle, plan.handle, _ptr(pt), _ptr(ct), _ptr(out), _ptr(ws),
                              ws.numel() * 8, mode, _stream()))
        return out

    def he_square(self, evk, ct, level):
        n = ct.shape[0]
        ws = self.workspace(load().fe_square_workspace_bytes(self.handle, n, level))
        out = self.empty_ct(n, level - 1)
        check(load().fe_he_square(self.handle, evk.handle, _ptr(ct), n, level, _ptr(out), _ptr(ws), ws.numel() * 8,
                                  _stream()))
        return out

    def he_avgpool(self, lay, ct, level):
        out_lay = FeLayout()
        n_out = lay.n_ct // 4
        out = self.empty_ct(n_out, level)
        check(load().fe_he_avgpool(self.handle, ctypes.byref(lay), _ptr(ct), level, _ptr(out),
                                   ctypes.byref(out_lay), _stream()))
        return out, out_lay

    def compress(self, evk, lay, c_valid, ct, level):
        n = ct.shape[0]
        ws = self.workspace(load().fe_compress_workspace_bytes(self.handle, n, level))
        out = self.empty_ct(n, level)
        check(load().fe_compress(self.handle, evk.handle, ctypes.byref(lay), c_valid, _ptr(ct), n, level, _ptr(out),
                                 _ptr(ws), ws.numel() * 8, _stream()))
        return out

    def graph_workspace_bytes(self, plans, n_req=1):
        n = len(plans)
        parr = (vp * n)(*[p.handle.value for p in plans])
        return int(load().fe_graph_workspace_bytes(parr, n, n_req))

    def graph_workspace_bytes_chunked(self, plans, n_req, req_chunk):
        n = len(plans)
        parr = (vp * n)(*[p.handle.value for p in plans])
        return int(load().fe_graph_workspace_bytes_chunked(parr, n, n_req, req_chunk))

    def graph_capture(self, evk, plans, pts, ins, outs, ws, n_req=1, req_chunk=None):
        n = len(plans)
        parr = (vp * n)(*[p.handle.value for p in plans])
        ptarr = (vp * n)(*[t.data_ptr() for t in pts])
        iarr = (vp * n)(*[t.data_ptr() for t in ins])
        oarr = (vp * n)(*[t.data_ptr() for t in outs])
        h = vp()
        if req_chunk is None:
            check(load().fe_graph_capture_batch(self.handle, evk.handle, parr, ptarr, iarr, oarr, n, n_req, _ptr(ws),
                                                ws.numel() * 8, _stream(), ctypes.byref(h)))
        else:
            check(load().fe_graph_capture_chunked(self.handle, evk.handle, parr, ptarr, iarr, oarr, n, n_req,
                                                  req_chunk, _ptr(ws), ws.numel() * 8, _stream(), ctypes.byref(h)))
        return Graph(h, (plans, pts, ins, outs, ws))

    def profile_begin(self, kind):
        check(load().fe_profile_begin(self.handle, kind.encode()))

    def profile_end(self):
        ms, n, b = dbl(), u64(), dbl()
        check(load().fe_profile_end(self.handle, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)))
        return ms.value, int(n.value), b.value

    # -- scale rule shared by the network code --------------------------------------------
    def weight_scale(self, level, s_in, delta, act_a=0.0):
        """fe_weight_scale: the weights' scale of a linear layer at `level` with input scale
        s_in (act_a: leading coefficient of the activation that follows, 0 for none)."""
        r = dbl()
        check(load().fe_weight_scale(self.handle, level, float(s_in), float(delta), float(act_a), ctypes.byref(r)))
        return r.value

    def plan_out_scale(self, plan, in_scale):
        """fe_plan_out_scale: output scale of a plan with loaded weights."""
        r = dbl()
        check(load().fe_plan_out_scale(plan.handle, float(in_scale), ctypes.byref(r)))
        return r.value

    def poly_act_scale(self, level, in_scale, a):
        r = dbl()
        check(load().fe_poly_act_scale(self.handle, level, float(in_scale), float(a), ctypes.byref(r)))
        return r.value

    def he_poly_act(self, evk, ct, level, in_scale, a, b, c):
        """a x^2 + b x + c on ciphertexts at `level` with scale in_scale; returns (out, out_scale)."""
        n = ct.shape[0]
        ws = self.workspace(load().fe_poly_act_workspace_bytes(self.handle, n, level))
        out = self.empty_ct(n, level - 1)
        sc = dbl()
        check(load().fe_he_poly_act(self.handle, evk.handle if evk is not None else None, float(a), float(b),
                                    float(c), _ptr(ct), n, level, float(in_scale), _ptr(out), ctypes.byref(sc),
                                    _ptr(ws), ws.numel() * 8, _stream()))
        return out, sc.value

    def compress_masked(self, evk, lay, c_valid, mask_scale, ct, level, in_scale):
        """AAC with its 0/1 mask at mask_scale; returns (out, out_scale)."""
        n = ct.shape[0]
        ws = self.workspace(load().fe_compress_masked_workspace_bytes(self.handle, n, level))
        out = self.empty_ct(n, level)
        sc = dbl()
        check(load().fe_compress_masked(self.handle, evk.handle, ctypes.byref(lay), c_valid, float(mask_scale),
                                        _ptr(ct), n, level, float(in_scale), _ptr(out), ctypes.byref(sc), _ptr(ws),
                                        ws.numel() * 8, _stream()))
        return out, sc.value

    def plan_fc_layout(self, lay, F_out, level):
        h = vp()
        check(load().fe_plan_fc_layout(self.handle, ctypes.byref(lay), F_out, level, ctypes.byref(h)))
        p = Plan(self, h)
        p.level = level
        return p

    def plan_repack(self, lay_from, lay_to, level):
        """fe_plan_repack: re-encoding from one fragment layout to another (one level)."""
        h = vp()
        check(load().fe_plan_repack(self.handle, ctypes.byref(lay_from), ctypes.byref(lay_to), level,
                                    ctypes.byref(h)))
        p = Plan(self, h, lay_to)
        p.level, p.in_layout = level, lay_from
        return p

    def load_repack_masks(self, plan, w_scale=None):
        """Encode a repack plan's masks (at q_level unless given)."""
        torch = _torch()
        w_scale = float(self.moduli[plan.level]) if w_scale is None else w_scale
        pt = torch.empty(max(8, plan.info.pt_bytes) // 8, dtype=torch.int64, device="cuda")
        check(load().fe_plan_load_weights(self.handle, plan.handle, None, 1.0, w_scale, _ptr(pt), _stream()))
        return pt

    def he_repack(self, evk, plan, pt, ct, mode=1, ws=None, out=None):
        ws = self.workspace(plan.info.workspace_bytes) if ws is None else ws
        out = self.empty_ct(plan.info.n_out_ct, plan.level - 1) if out is None else out
        self._check_layer_buffers(plan, pt, ct, out)
        check(load().fe_he_repack(self.handle, evk.handle, plan.handle, _ptr(pt), _ptr(ct), _ptr(out), _ptr(ws),
                                  ws.numel() * 8, mode, _stream()))
        return out

    def token_layout(self, n_tok, E, S):
        lay = FeTokenLayout(n_tok, E, S, 0, 0, 0)
        check(load().fe_token_layout_make(self.handle, ctypes.byref(lay)))
        return lay

    def token_pack(self, lay, x):
        torch = _torch()
        x = torch.as_tensor(x, dtype=torch.float64).cuda().contiguous()
        slots = torch.empty((lay.n_ct, self.N // 2), dtype=torch.float64, device="cuda")
        check(load().fe_token_pack(self.handle, ctypes.byref(lay), _ptr(x), _ptr(slots), _stream()))
        return slots

    def token_unpack(self, lay, slots):
        torch = _torch()
        x = torch.zeros((lay.n_tok, lay.E), dtype=torch.float64, device="cuda")
        check(load().fe_token_unpack(self.handle, ctypes.byref(lay), _ptr(slots.contiguous()), _ptr(x), _stream()))
        return x

    def plan_token_linear(self, lay, E_out, level):
        out_lay = FeTokenLayout()
        h = vp()
        check(load().fe_plan_token_linear(self.handle, ctypes.byref(lay), E_out, level, ctypes.byref(out_lay),
                                          ctypes.byref(h)))
        p = Plan(self, h)
        p.level, p.token_out = level, out_lay
        return p

    def attention_rotation_steps(self, lay):
        n = u32()
        check(load().fe_attention_rotation_steps(self.handle, ctypes.byref(lay), None, 0, ctypes.byref(n)))
        arr = (i32 * max(1, n.value))()
        check(load().fe_attention_rotation_steps(self.handle, ctypes.byref(lay), arr, n.value, ctypes.byref(n)))
        return [arr[i] for i in range(n.value)]

    def he_attention_scores(self, evk, lay, q, k, level, q_scale, k_scale):
        """Diagonals of Q K^T: returns (out [n_tok, 2, level-1, N], out_scale)."""
        for t in (q, k):
            if t.numel() != lay.n_ct * self.ct_words(level):
                raise ValueError("Q and K must hold S ciphertexts at `level`")
        out = self.empty_ct(lay.n_tok, level - 2)
        sc = dbl()
        check(load().fe_he_attention_scores(self.handle, evk.handle, ctypes.byref(lay), _ptr(q), _ptr(k), level,
                                            float(q_scale), float(k_scale), _ptr(out), ctypes.byref(sc), _stream()))
        return out, sc.value

    def he_attention_apply(self, evk, lay, d, d_level, d_scale, v, v_level, v_scale):
        """(Q K^T) V from the score diagonals: returns (out, out_level, out_scale)."""
        if d.numel() != lay.n_tok * self.ct_words(d_level) or v.numel() != lay.n_ct * self.ct_words(v_level):
            raise ValueError("D must hold n_tok ciphertexts at d_level, V S at v_level")
        ml = min(v_level - 1, d_level)
        out = self.empty_ct(lay.n_ct, ml - 1)
        lv, sc = u32(), dbl()
        check(load().fe_he_attention_apply(self.handle, evk.handle, ctypes.byref(lay), _ptr(d), d_level,
                                           float(d_scale), _ptr(v), v_level, float(v_scale), _ptr(out),
                                           ctypes.byref(lv), ctypes.byref(sc), _stream()))
        return out, lv.value, sc.value

    def plan_fc_next(self, prev, F_out, level):
        h = vp()
        check(load().fe_plan_fc_next(self.handle, prev.handle, F_out, level, ctypes.byref(h)))
        p = Plan(self, h)
        p.level = level
        return p

    def fc_unpack(self, plan, slots, BS, F_out):
        """fe_fc_unpack: decoded output slots of an FC plan -> (BS, F_out) outputs."""
        torch = _torch()
        y = torch.empty((BS, F_out), dtype=torch.float64, device="cuda")
        check(load().fe_fc_unpack(self.handle, plan.handle, _ptr(slots.contiguous()), _ptr(y), _stream()))
        return y


P_i32 = ctypes.POINTER(i32)


class MLP:
    """fp32 latency model (in_dim -> hidden x n_hidden ReLU -> 1) with CUDA
    training (full-batch Adam) and inference kernels."""

    def __init__(self, in_dim, hidden=64, n_hidden=3, seed=0):
        h = vp()
        check(load().fe_mlp_create(in_dim, hidden, n_hidden, seed, ctypes.byref(h)))
        self.handle = h
        self.in_dim, self.hidden, self.n_hidden = in_dim, hidden, n_hidden

    def params(self):
        n = load().fe_mlp_param_count(self.handle)
        a = np.zeros(n, dtype=np.float32)
        check(load().fe_mlp_get_params(self.handle, a.ctypes.data_as(P(ctypes.c_float))))
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        assert a.size == load().fe_mlp_param_count(self.handle)
        check(load().fe_mlp_set_params(self.handle, a.ctypes.data_as(P(ctypes.c_float))))

    def scaling(self):
        xm = np.zeros(self.in_dim, np.float32)
        xs = np.zeros(self.in_dim, np.float32)
        ys = np.zeros(2, np.float32)
        fp = P(ctypes.c_float)
        check(load().fe_mlp_get_scaling(self.handle, xm.ctypes.data_as(fp), xs.ctypes.data_as(fp),
                                        ys.ctypes.data_as(fp)))
        return xm, xs, ys

    def train(self, X, y, steps=2000, lr=1e-3, weight_decay=0.0):
        torch = _torch()
        Xd = torch.as_tensor(np.ascontiguousarray(X, np.float32)).cuda()
        yd = torch.as_tensor(np.ascontiguousarray(y, np.float32)).cuda()
        loss = ctypes.c_float(0)
        check(load().fe_mlp_train(self.handle, _ptr(Xd), _ptr(yd), Xd.shape[0], steps, lr, weight_decay,
                                  ctypes.byref(loss), _stream()))
        return loss.value

    def predict(self, X):
        torch = _torch()
        Xd = torch.as_tensor(np.ascontiguousarray(X, np.float32)).cuda()
        yd = torch.empty(Xd.shape[0], dtype=torch.float32, device="cuda")
        check(load().fe_mlp_predict(self.handle, _ptr(Xd), Xd.shape[0], _ptr(yd), _stream()))
        return yd.cpu().numpy()

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fe_mlp_destroy(self.handle)
            self.handle = None


class Server:
    """Request loop over registered models (continuous batching, admission by
    device memory, resident keys).  Plans, plaintexts, keys and contexts passed
    to add_model must outlive the server; host buffers passed to submit must
    stay alive until the request finishes."""

    def __init__(self, max_batch=4, max_inflight=3, hbm_budget_bytes=0, hbm_reserve_bytes=4 << 30):
        cfg = FeServerConfig(max_batch, max_inflight, hbm_budget_bytes, hbm_reserve_bytes)
        h = vp()
        check(load().fe_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self._keep = []

    def add_model(self, ctx, evk, ops, in_ct, in_level):
        """ops: list of (OP_LAYER, plan, pt) / (OP_SQUARE,) / (OP_POOL, layout) /
        (OP_POLY_ACT, a, b, c, in_scale) / (OP_REFRESH, boot, in_scale)."""
        arr = (FeOp * len(ops))()
        for i, op in enumerate(ops):
            if op[0] == OP_LAYER:
                arr[i] = FeOp(OP_LAYER, op[1].handle, _ptr(op[2]), FeLayout())
            elif op[0] == OP_SQUARE:
                arr[i] = FeOp(OP_SQUARE, None, None, FeLayout())
            elif op[0] == OP_POLY_ACT:
                arr[i] = FeOp(OP_POLY_ACT, None, None, FeLayout(), float(op[1]), float(op[2]), float(op[3]),
                              float(op[4]), None)
            elif op[0] == OP_REFRESH:
                arr[i] = FeOp(OP_REFRESH, None, None, FeLayout(), 0.0, 0.0, 0.0, float(op[2]), op[1].handle)
            else:
                arr[i] = FeOp(OP_POOL, None, None, op[1])
        mid = u32(0)
        check(load().fe_server_add_model(self.handle, ctx.handle, evk.handle, arr, len(ops), in_ct, in_level,
                                         ctypes.byref(mid)))
        self._keep.append((ctx, evk, ops))
        return mid.value

    def model_io(self, model):
        oc, ol, ib, ob = u32(0), u32(0), sz(0), sz(0)
        check(load().fe_server_model_io(self.handle, model, ctypes.byref(oc), ctypes.byref(ol), ctypes.byref(ib),
                                        ctypes.byref(ob)))
        return oc.value, ol.value, ib.value, ob.value

    def pause(self, paused=True):
        check(load().fe_server_pause(self.handle, 1 if paused else 0))

    def submit(self, model, in_host, out_host):
        rid = u64(0)
        check(load().fe_server_submit(self.handle, model, _ptr(in_host), _ptr(out_host), ctypes.byref(rid)))
        return rid.value

    def wait(self, rid, timeout_ms=600000):
        st, lat = cint(0), dbl(0)
        check(load().fe_server_wait(self.handle, rid, timeout_ms, ctypes.byref(st), ctypes.byref(lat)))
        return st.value, lat.value

    def stats(self):
        r = FeServerStats()
        check(load().fe_server_stats(self.handle, ctypes.byref(r)))
        return r.as_dict()

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fe_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def rotation_model(N, H, W, Cin, Cout, K, S, BS, stride=1, depthwise=False):
    """Eq. 3 - Eq. 8 counts of one conv layer at fragment size S (host only)."""
    r = FeRotationModel()
    check(load().fe_rotation_model(N, H, W, Cin, Cout, K, S, BS, stride, 1 if depthwise else 0, ctypes.byref(r)))
    return r.as_dict()


def choose_fragment(N, H, W, Cin, Cout, K, BS, depthwise=False, max_S=0):
    """Analytic fragment-size choice: argmin of Eq. 5 over admissible S (host only)."""
    r = FeFragmentChoice()
    check(load().fe_choose_fragment(N, H, W, Cin, Cout, K, BS, 1 if depthwise else 0, max_S, ctypes.byref(r)))
    return r.as_dict()


def choose_token_fragment(E, n_tok, gamma, max_S=0):
    """Block size of the transformer extension: argmin of gamma E / S + 2 n S (host only)."""
    S, r, st = u32(0), dbl(), dbl()
    check(load().fe_choose_token_fragment(E, n_tok, float(gamma), max_S, ctypes.byref(S), ctypes.byref(r),
                                          ctypes.byref(st)))
    return {"S": S.value, "rotations": r.value, "s_star": st.value}


def exported_symbols():
    """Names of the C ABI entry points this binding expects the library to export."""
    return sorted(SIGNATURES)
