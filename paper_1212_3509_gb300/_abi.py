"""ctypes binding of libdemag (include/demag.h).

Argument marshalling only: every step of the operator runs in the CUDA
library.  Functions carry the C names; tensors are PyTorch CUDA tensors of
the documented dtype and size (contiguous), or raw integer device pointers.
The library must have been built (``paper_1212_3509_gb300.build.build()``);
importing this module without it raises immediately.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libdemag.so")

PRECISIONS = {"fp64": 0, "fp32": 1, "tf32x3": 2, "bf16x3": 3}
STATUS = {0: "DEMAG_OK", 1: "DEMAG_EINVAL", 2: "DEMAG_ENOMEM", 3: "DEMAG_ECUDA",
          4: "DEMAG_ETIMEOUT", 5: "DEMAG_EUNSUPPORTED"}


class DemagError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("h", ctypes.c_double * 3), ("R", ctypes.c_int), ("c0", ctypes.c_double)]


class GridEdgesDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("edges", ctypes.POINTER(ctypes.c_double) * 3), ("R", ctypes.c_int),
                ("c0", ctypes.c_double)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libdemag is not built ({LIB_PATH} missing); run paper_1212_3509_gb300.build.build()")

lib = ctypes.CDLL(LIB_PATH)

_vp, _i, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
_SIGS = {
    "demag_build_factors": (_i, [ctypes.POINTER(GridDesc), ctypes.POINTER(_vp), _vp]),
    "demag_plan_destroy": (None, [_vp]),
    "demag_num_terms": (_i, [_vp]),
    "demag_last_error": (ctypes.c_char_p, [_vp]),
    "demag_copy_nodes": (_i, [_vp, _vp, _vp]),
    "demag_copy_generators": (_i, [_vp, _vp, _vp]),
    "demag_copy_symbols": (_i, [_vp, _vp, _vp]),
    "demag_generators_size": (_sz, [_vp]),
    "demag_symbols_size": (_sz, [_vp]),
    "demag_apply_full": (_i, [_vp, _vp, _vp, _i, _vp]),
    "demag_apply_full_fft": (_i, [_vp, _vp, _vp, _vp]),
    "demag_apply_full_fibres": (_i, [_vp, _vp, _vp, _vp]),
    "demag_stray_field_fft": (_i, [_vp, _vp, _vp, _vp]),
    "demag_energy_field_fft": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "demag_build_factors_nonuniform": (_i, [ctypes.POINTER(GridEdgesDesc), ctypes.POINTER(_vp), _vp]),
    "demag_compress_kernel": (_i, [_vp, ctypes.c_double, _vp]),
    "demag_compressed_ranks": (_i, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "demag_copy_compressed": (_i, [_vp, _vp, _vp, _vp]),
    "demag_apply_tucker_compressed": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_int), _vp, _vp, _vp, _vp, _vp]),
    "demag_recompress_tucker": (_i, [_vp, ctypes.POINTER(ctypes.c_int), _vp, _vp, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_int), _vp, _vp, ctypes.POINTER(ctypes.c_double), _vp]),
    "demag_tucker_to_tt": (_i, [_vp, ctypes.POINTER(_i), _vp, _vp, _vp, _vp, _vp, _vp]),
    "demag_cp_to_tt": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
    "demag_tt_hadamard": (_i, [_vp, ctypes.POINTER(_i), _vp, _vp, _vp, ctypes.POINTER(_i), _vp, _vp, _vp, _vp, _vp,
                               _vp, _vp]),
    "demag_round_tt": (_i, [_vp, ctypes.POINTER(ctypes.c_int), _vp, _vp, _vp, _vp, ctypes.c_double,
                            ctypes.POINTER(ctypes.c_int), _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double), _vp]),
    "demag_apply_full_batched": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _i, _vp]),
    "demag_graph_create_batched": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _i,
                                        ctypes.POINTER(_vp)]),
    "demag_graph_launch": (_i, [_vp, _vp]),
    "demag_graph_kernel_count": (_i, [_vp]),
    "demag_graph_destroy": (None, [_vp]),
    "demag_reserve_workspace": (_i, [_vp, _i]),
    "demag_apply_adjoint": (_i, [_vp, _vp, _vp, _i, _vp]),
    "demag_apply_cp": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp]),
    "demag_apply_cp_batched": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp, _vp]),
    "demag_apply_tucker": (_i, [_vp, ctypes.POINTER(_i), _vp, _vp, _vp, _vp]),
    "demag_apply_tt": (_i, [_vp, ctypes.POINTER(_i), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "demag_apply_tucker_batched": (_i, [_vp, _i, ctypes.POINTER(_i), _vp, _vp, _vp, _vp]),
    "demag_apply_tt_batched": (_i, [_vp, _i, ctypes.POINTER(_i), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "demag_energy_tucker": (_i, [_vp, ctypes.POINTER(_i), _vp, _vp, _vp, _vp, _vp, _vp]),
    "demag_energy_tt": (_i, [_vp, ctypes.POINTER(_i), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "demag_energy_tucker_phi": (_i, [_vp, ctypes.POINTER(_i), _vp, _vp, ctypes.POINTER(_i), _vp, _vp, _vp, _vp]),
    "demag_energy_tucker_fp64": (_i, [_vp, ctypes.POINTER(_i), _vp, _vp, _vp, _vp]),
    "demag_stray_field": (_i, [_vp, _vp, _vp, _vp]),
    "demag_stray_field_exact": (_i, [_vp, _vp, _vp, _i, _vp]),
    "demag_energy": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
    "demag_sync_status": (_i, [_vp, _vp]),
    "demag_apply_full_noalloc": (_i, [ctypes.POINTER(GridDesc), _vp, _vp, _vp]),
    "demag_launch_count": (ctypes.c_ulonglong, [_vp]),
    "demag_autotune": (_i, [_vp, _i]),
    "demag_set_wait_limit": (_i, [_vp, ctypes.c_double]),
    "demag_set_fused": (_i, [_vp, ctypes.c_int]),
    "demag_forward_schedule": (_i, [_vp, ctypes.c_int]),
    "demag_autotune_count": (_i, [_vp]),
    "demag_autotune_entry": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    "demag_autotune_save": (_i, [_vp, ctypes.c_char_p]),
    "demag_autotune_load": (_i, [_vp, ctypes.c_char_p, ctypes.POINTER(_i)]),
    "demag_profile": (_i, [_vp, _i]),
    "demag_profile_read": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "demag_profile_count": (ctypes.c_longlong, [_vp]),
    "demag_profile_launch": (_i, [_vp, ctypes.c_longlong, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_double)]),
}

FAMILIES = {"gemm_simt": 0, "gemm_tc": 1, "fft": 2, "split": 3, "setup": 4, "energy": 5, "misc": 6,
            "fft3d": 7}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _check(status: int, plan_ptr=None):
    if status != 0:
        msg = lib.demag_last_error(plan_ptr).decode(errors="replace")
        raise DemagError(status, msg)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t, numel=None, dtype=None, name="tensor"):
    """Device pointer of a tensor (validated) or an int passed through."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    import torch
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


def _prec(p):
    if isinstance(p, int):
        return p
    return PRECISIONS[p.lower()]


class Plan:
    """Owns a demag_plan*.  Attributes mirror demag_grid_desc; M = (R-1)/2."""

    def __init__(self, ptr: int, n, h, R: int, c0: float):
        self.ptr = ptr
        self.n = tuple(int(v) for v in n)
        self.h = tuple(float(v) for v in h)
        self.R, self.c0 = int(R), float(c0)
        self.M = lib.demag_num_terms(ptr)

    @property
    def N(self):
        return self.n[0] * self.n[1] * self.n[2]

    def close(self):
        if self.ptr:
            lib.demag_plan_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def demag_build_factors(n, h, R: int, c0: float = 2.15, stream=None) -> Plan:
    d = GridDesc((ctypes.c_int * 3)(*[int(v) for v in n]), (ctypes.c_double * 3)(*[float(v) for v in h]), int(R), float(c0))
    out = _vp()
    _check(lib.demag_build_factors(ctypes.byref(d), ctypes.byref(out), _stream(stream)))
    return Plan(out.value, n, h, R, c0)


def demag_build_factors_nonuniform(edges, R: int, c0: float = 2.15, stream=None) -> Plan:
    """Plan for a non-uniform tensor grid: edges[p] = the n_p + 1 increasing cell edges of axis p (i1 first)."""
    arrs = [(ctypes.c_double * len(e))(*[float(v) for v in e]) for e in edges]
    if len(arrs) != 3 or any(len(a) < 2 for a in arrs):
        raise ValueError("edges: three arrays of at least two cell edges")
    n = [len(a) - 1 for a in arrs]
    d = GridEdgesDesc((ctypes.c_int * 3)(*n),
                      (ctypes.POINTER(ctypes.c_double) * 3)(*[ctypes.cast(a, ctypes.POINTER(ctypes.c_double))
                                                              for a in arrs]),
                      int(R), float(c0))
    out = _vp()
    _check(lib.demag_build_factors_nonuniform(ctypes.byref(d), ctypes.byref(out), _stream(stream)))
    mean_h = [(float(e[-1]) - float(e[0])) / (len(e) - 1) for e in edges]
    plan = Plan(out.value, n, mean_h, R, c0)
    plan.edges = [tuple(float(v) for v in e) for e in edges]
    return plan


def demag_compress_kernel(plan: Plan, tol: float, stream=None):
    """Alg. 2 setup: compress the three CP kernels to Tucker tensors (HOOI, tolerance tol)."""
    _check(lib.demag_compress_kernel(plan.ptr, float(tol), _stream(stream)), plan.ptr)


def demag_compressed_ranks(plan: Plan) -> tuple:
    rho = (ctypes.c_int * 3)()
    _check(lib.demag_compressed_ranks(plan.ptr, rho), plan.ptr)
    return tuple(int(v) for v in rho)


def demag_copy_compressed(plan: Plan, gen=None, core=None, stream=None):
    import torch
    rho = demag_compressed_ranks(plan)
    glen = 2 * max(plan.n) - 1
    _check(lib.demag_copy_compressed(plan.ptr, _ptr(gen, max(rho) * 9 * glen, torch.float64, "gen"),
                                     _ptr(core, 3 * rho[0] * rho[1] * rho[2], torch.float32, "core"),
                                     _stream(stream)), plan.ptr)


def demag_apply_tucker_compressed(plan: Plan, batch: int, r, core, V, out_core, out_V, stream=None):
    import torch
    rho = demag_compressed_ranks(plan)
    rr = (ctypes.c_int * 3)(*[int(v) for v in r])
    f32 = torch.float32
    qs = sum(int(r[p]) * plan.n[p] for p in range(3))
    os_ = sum(3 * rho[p] * int(r[p]) * plan.n[p] for p in range(3))
    ncore = int(r[0]) * int(r[1]) * int(r[2])
    nout = rho[0] * r[0] * rho[1] * r[1] * rho[2] * r[2]
    _check(lib.demag_apply_tucker_compressed(plan.ptr, int(batch), rr,
                                             _ptr(core, batch * 3 * ncore, f32, "core"),
                                             _ptr(V, batch * 3 * qs, f32, "V"),
                                             _ptr(out_core, batch * 3 * nout, f32, "out_core"),
                                             _ptr(out_V, batch * os_, f32, "out_V"), _stream(stream)), plan.ptr)


def _tt_sizes(plan: Plan, r1: int, r2: int):
    return 3 * r1 * plan.n[0], 3 * r1 * r2 * plan.n[1], 3 * r2 * plan.n[2]


def demag_tucker_to_tt(plan: Plan, ranks, core, V, G1, G2, G3, stream=None):
    """Tucker magnetization -> trains of ranks (r1, r3) (App. C)."""
    import torch
    r = (_i * 3)(*[int(v) for v in ranks])
    f32 = torch.float32
    s1, s2, s3 = _tt_sizes(plan, int(ranks[0]), int(ranks[2]))
    tot = sum(int(ranks[p]) * plan.n[p] for p in range(3))
    _check(lib.demag_tucker_to_tt(plan.ptr, r, _ptr(core, 3 * int(ranks[0]) * int(ranks[1]) * int(ranks[2]), f32,
                                                    "core"),
                                  _ptr(V, 3 * tot, f32, "V"), _ptr(G1, s1, f32, "G1"), _ptr(G2, s2, f32, "G2"),
                                  _ptr(G3, s3, f32, "G3"), _stream(stream)), plan.ptr)


def demag_cp_to_tt(plan: Plan, r: int, lam, U, G1, G2, G3, stream=None):
    """CP magnetization -> trains of ranks (r, r) with a diagonal middle core (App. C)."""
    import torch
    f32 = torch.float32
    s1, s2, s3 = _tt_sizes(plan, int(r), int(r))
    _check(lib.demag_cp_to_tt(plan.ptr, int(r), _ptr(lam, 3 * int(r), f32, "lambda"),
                              _ptr(U, 3 * int(r) * sum(plan.n), f32, "U"), _ptr(G1, s1, f32, "G1"),
                              _ptr(G2, s2, f32, "G2"), _ptr(G3, s3, f32, "G3"), _stream(stream)), plan.ptr)


def demag_tt_hadamard(plan: Plan, ra, A, rb, B, C, stream=None):
    """C = A .* B per component; A, B, C are (G1, G2, G3) triples; C has ranks (ra1 rb1, ra2 rb2)."""
    import torch
    f32 = torch.float32
    a = (_i * 2)(int(ra[0]), int(ra[1]))
    b = (_i * 2)(int(rb[0]), int(rb[1]))
    sa = _tt_sizes(plan, int(ra[0]), int(ra[1]))
    sb = _tt_sizes(plan, int(rb[0]), int(rb[1]))
    sc = _tt_sizes(plan, int(ra[0]) * int(rb[0]), int(ra[1]) * int(rb[1]))
    _check(lib.demag_tt_hadamard(plan.ptr, a, *[_ptr(A[i], sa[i], f32, f"A{i + 1}") for i in range(3)], b,
                                 *[_ptr(B[i], sb[i], f32, f"B{i + 1}") for i in range(3)],
                                 *[_ptr(C[i], sc[i], f32, f"C{i + 1}") for i in range(3)], _stream(stream)), plan.ptr)


def demag_round_tt(plan: Plan, r, w, o1, o2, o3, tol: float, stream=None):
    """Round one item's TT output (demag_apply_tt): returns ((r1, r2), G1 [r1, n1], G2 [r1 r2, n2], G3 [r2, n3], err)."""
    import torch
    n1, n2, n3 = plan.n
    r1, r2 = int(r[0]), int(r[1])
    M = plan.M
    f32 = torch.float32
    rr = (ctypes.c_int * 2)(r1, r2)
    G1o = torch.empty(64 * n1, device="cuda")
    G2o = torch.empty(64 * 64 * n2, device="cuda")
    G3o = torch.empty(64 * n3, device="cuda")
    ranks = (ctypes.c_int * 2)()
    err = ctypes.c_double()
    _check(lib.demag_round_tt(plan.ptr, rr, _ptr(w, 3 * M, f32, "w"), _ptr(o1, 3 * M * r1 * n1, f32, "o1"),
                              _ptr(o2, 3 * M * r1 * r2 * n2, f32, "o2"), _ptr(o3, 3 * M * r2 * n3, f32, "o3"),
                              float(tol), ranks, G1o.data_ptr(), G2o.data_ptr(), G3o.data_ptr(), ctypes.byref(err),
                              _stream(stream)), plan.ptr)
    q1, q2 = int(ranks[0]), int(ranks[1])
    return ((q1, q2), G1o[: q1 * n1].reshape(q1, n1), G2o[: q1 * q2 * n2].reshape(q1 * q2, n2),
            G3o[: q2 * n3].reshape(q2, n3), err.value)


def demag_recompress_tucker(plan: Plan, r, core, V, tol: float, stream=None):
    """Recompress one item's compressed Tucker output: returns (ranks, core [r3, r2, r1], [U_p [r_p, n_p]], err)."""
    import torch
    rho = demag_compressed_ranks(plan)
    rr = (ctypes.c_int * 3)(*[int(v) for v in r])
    f32 = torch.float32
    nv = sum(3 * rho[p] * int(r[p]) * plan.n[p] for p in range(3))
    core_out = torch.empty(64 ** 3, device="cuda")
    U_out = torch.empty(64 * sum(plan.n), device="cuda")
    ranks = (ctypes.c_int * 3)()
    err = ctypes.c_double()
    _check(lib.demag_recompress_tucker(plan.ptr, rr, _ptr(core, 3 * int(r[0]) * int(r[1]) * int(r[2]), f32, "core"),
                                       _ptr(V, nv, f32, "V"), float(tol), ranks, core_out.data_ptr(),
                                       U_out.data_ptr(), ctypes.byref(err), _stream(stream)), plan.ptr)
    rk = tuple(int(v) for v in ranks)
    C = core_out[: rk[0] * rk[1] * rk[2]].reshape(rk[2], rk[1], rk[0])
    Us, off = [], 0
    for p in range(3):
        Us.append(U_out[off: off + rk[p] * plan.n[p]].reshape(rk[p], plan.n[p]))
        off += rk[p] * plan.n[p]
    return rk, C, Us, err.value


def demag_plan_destroy(plan: Plan):
    plan.close()


def demag_num_terms(plan: Plan) -> int:
    return lib.demag_num_terms(plan.ptr)


def demag_last_error(plan: Plan | None = None) -> str:
    return lib.demag_last_error(plan.ptr if plan else None).decode(errors="replace")


def demag_generators_size(plan: Plan) -> int:
    return lib.demag_generators_size(plan.ptr)


def demag_symbols_size(plan: Plan) -> int:
    return lib.demag_symbols_size(plan.ptr)


def demag_copy_nodes(plan: Plan, dst, stream=None):
    import torch
    _check(lib.demag_copy_nodes(plan.ptr, _ptr(dst, 3 * plan.M, torch.float64, "dst"), _stream(stream)), plan.ptr)


def demag_copy_generators(plan: Plan, dst, stream=None):
    import torch
    _check(lib.demag_copy_generators(plan.ptr, _ptr(dst, demag_generators_size(plan), torch.float64, "dst"),
                                     _stream(stream)), plan.ptr)


def demag_copy_symbols(plan: Plan, dst, stream=None):
    import torch
    _check(lib.demag_copy_symbols(plan.ptr, _ptr(dst, demag_symbols_size(plan), torch.float32, "dst"),
                                  _stream(stream)), plan.ptr)


def demag_apply_full(plan: Plan, m, phi, precision="fp32", stream=None):
    import torch
    _check(lib.demag_apply_full(plan.ptr, _ptr(m, 3 * plan.N, torch.float32, "m"),
                                _ptr(phi, plan.N, torch.float32, "phi"), _prec(precision), _stream(stream)), plan.ptr)


def demag_apply_full_fft(plan: Plan, m, phi, stream=None):
    import torch
    _check(lib.demag_apply_full_fft(plan.ptr, _ptr(m, 3 * plan.N, torch.float32, "m"),
                                    _ptr(phi, plan.N, torch.float32, "phi"), _stream(stream)), plan.ptr)


def demag_apply_full_fibres(plan: Plan, m, phi, stream=None):
    import torch
    _check(lib.demag_apply_full_fibres(plan.ptr, _ptr(m, 3 * plan.N, torch.float32, "m"),
                                       _ptr(phi, plan.N, torch.float32, "phi"), _stream(stream)), plan.ptr)


def demag_stray_field_fft(plan: Plan, m, hd, stream=None):
    import torch
    _check(lib.demag_stray_field_fft(plan.ptr, _ptr(m, 3 * plan.N, torch.float32, "m"),
                                     _ptr(hd, 3 * plan.N, torch.float32, "hd"), _stream(stream)), plan.ptr)


def demag_energy_field_fft(plan: Plan, m, energy, grad=None, stream=None):
    import torch
    _check(lib.demag_energy_field_fft(plan.ptr, _ptr(m, 3 * plan.N, torch.float32, "m"),
                                      _ptr(energy, 1, torch.float64, "energy"),
                                      _ptr(grad, 3 * plan.N, torch.float32, "grad"), _stream(stream)), plan.ptr)


def demag_apply_full_batched(plans, ms, phis, precision="bf16x3", stream=None):
    cnt, P, Mp, Fp = _batch_arrays(plans, ms, phis)
    _check(lib.demag_apply_full_batched(P, Mp, Fp, cnt, _prec(precision), _stream(stream)))


def _batch_arrays(plans, ms, phis):
    import torch
    cnt = len(plans)
    P = (_vp * cnt)(*[p.ptr for p in plans])
    Mp = (_vp * cnt)(*[_ptr(m, 3 * p.N, torch.float32, "m") for m, p in zip(ms, plans)])
    Fp = (_vp * cnt)(*[_ptr(f, p.N, torch.float32, "phi") for f, p in zip(phis, plans)])
    return cnt, P, Mp, Fp


class Graph:
    """Owns a demag_graph* (a captured batched apply).  Keeps the plans and
    tensors it was recorded with alive while it exists."""

    def __init__(self, ptr: int, plans, ms, phis):
        self.ptr = ptr
        self._keep = (list(plans), list(ms), list(phis))
        self.kernels = lib.demag_graph_kernel_count(ptr)

    def launch(self, stream=None):
        demag_graph_launch(self, stream)

    def close(self):
        if self.ptr:
            lib.demag_graph_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def demag_graph_create_batched(plans, ms, phis, precision="bf16x3") -> Graph:
    cnt, P, Mp, Fp = _batch_arrays(plans, ms, phis)
    out = _vp()
    _check(lib.demag_graph_create_batched(P, Mp, Fp, cnt, _prec(precision), ctypes.byref(out)))
    return Graph(out.value, plans, ms, phis)


def demag_graph_launch(graph: Graph, stream=None):
    _check(lib.demag_graph_launch(graph.ptr, _stream(stream)))


def demag_graph_kernel_count(graph: Graph) -> int:
    return lib.demag_graph_kernel_count(graph.ptr)


def demag_graph_destroy(graph: Graph):
    graph.close()


def demag_reserve_workspace(plan: Plan, precision="fp32"):
    _check(lib.demag_reserve_workspace(plan.ptr, _prec(precision)), plan.ptr)


def demag_apply_adjoint(plan: Plan, y, g, precision="fp32", stream=None):
    import torch
    _check(lib.demag_apply_adjoint(plan.ptr, _ptr(y, plan.N, torch.float32, "y"),
                                   _ptr(g, 3 * plan.N, torch.float32, "g"), _prec(precision), _stream(stream)), plan.ptr)


def demag_apply_cp(plan: Plan, r: int, lam, U, out_w, out_U, stream=None):
    demag_apply_cp_batched(plan, 1, r, lam, U, out_w, out_U, stream)


def demag_apply_cp_batched(plan: Plan, batch: int, r: int, lam, U, out_w, out_U, stream=None):
    import torch
    ns = sum(plan.n)
    f32 = torch.float32
    _check(lib.demag_apply_cp_batched(plan.ptr, int(batch), int(r), _ptr(lam, batch * 3 * r, f32, "lambda"),
                                      _ptr(U, batch * 3 * r * ns, f32, "U"),
                                      _ptr(out_w, batch * plan.M * 3 * r, f32, "out_w"),
                                      _ptr(out_U, batch * plan.M * 3 * r * ns, f32, "out_U"), _stream(stream)), plan.ptr)


def demag_apply_tucker(plan: Plan, ranks, V, out_w, out_V, stream=None):
    demag_apply_tucker_batched(plan, 1, ranks, V, out_w, out_V, stream)


def demag_apply_tucker_batched(plan: Plan, batch: int, ranks, V, out_w, out_V, stream=None):
    import torch
    r = (_i * 3)(*[int(v) for v in ranks])
    tot = sum(int(ranks[p]) * plan.n[p] for p in range(3))
    f32, b = torch.float32, int(batch)
    _check(lib.demag_apply_tucker_batched(plan.ptr, b, r, _ptr(V, b * 3 * tot, f32, "V"),
                                          _ptr(out_w, b * plan.M * 3, f32, "out_w"),
                                          _ptr(out_V, b * plan.M * 3 * tot, f32, "out_V"), _stream(stream)), plan.ptr)


def demag_apply_tt(plan: Plan, ranks, G1, G2, G3, out_w, oG1, oG2, oG3, stream=None):
    demag_apply_tt_batched(plan, 1, ranks, G1, G2, G3, out_w, oG1, oG2, oG3, stream)


def demag_apply_tt_batched(plan: Plan, batch: int, ranks, G1, G2, G3, out_w, oG1, oG2, oG3, stream=None):
    import torch
    r1, r2 = int(ranks[0]), int(ranks[1])
    n1, n2, n3 = plan.n
    M, b = plan.M, int(batch)
    f32 = torch.float32
    r = (_i * 2)(r1, r2)
    _check(lib.demag_apply_tt_batched(plan.ptr, b, r, _ptr(G1, b * 3 * r1 * n1, f32, "G1"),
                                      _ptr(G2, b * 3 * r1 * r2 * n2, f32, "G2"),
                                      _ptr(G3, b * 3 * r2 * n3, f32, "G3"), _ptr(out_w, b * M * 3, f32, "out_w"),
                                      _ptr(oG1, b * M * 3 * r1 * n1, f32, "oG1"),
                                      _ptr(oG2, b * M * 3 * r1 * r2 * n2, f32, "oG2"),
                                      _ptr(oG3, b * M * 3 * r2 * n3, f32, "oG3"), _stream(stream)), plan.ptr)


def demag_stray_field(plan: Plan, phi, hd, stream=None):
    import torch
    _check(lib.demag_stray_field(plan.ptr, _ptr(phi, plan.N, torch.float32, "phi"),
                                 _ptr(hd, 3 * plan.N, torch.float32, "hd"), _stream(stream)), plan.ptr)


def demag_energy(plan: Plan, m, energy, grad=None, precision="fp32", stream=None):
    import torch
    _check(lib.demag_energy(plan.ptr, _ptr(m, 3 * plan.N, torch.float32, "m"), _ptr(energy, 1, torch.float64, "energy"),
                            _ptr(grad, 3 * plan.N, torch.float32, "grad"), _prec(precision), _stream(stream)), plan.ptr)


def demag_energy_tucker(plan: Plan, ranks, core, V, out_w, out_V, energy, stream=None):
    """Energy of a Tucker magnetization from its demag_apply_tucker output (energy: device float64)."""
    import torch
    r = (_i * 3)(*[int(v) for v in ranks])
    tot = sum(int(ranks[p]) * plan.n[p] for p in range(3))
    f32 = torch.float32
    _check(lib.demag_energy_tucker(plan.ptr, r, _ptr(core, 3 * int(ranks[0]) * int(ranks[1]) * int(ranks[2]), f32,
                                                     "core"),
                                   _ptr(V, 3 * tot, f32, "V"), _ptr(out_w, plan.M * 3, f32, "out_w"),
                                   _ptr(out_V, plan.M * 3 * tot, f32, "out_V"),
                                   _ptr(energy, 1, torch.float64, "energy"), _stream(stream)), plan.ptr)


def demag_energy_tucker_fp64(plan: Plan, ranks, core, V, energy, stream=None):
    """Energy of a Tucker magnetization with its Tucker application in FP64 (core, V, energy:
    device float64)."""
    import torch
    r = (_i * 3)(*[int(v) for v in ranks])
    tot = sum(int(ranks[p]) * plan.n[p] for p in range(3))
    f64 = torch.float64
    _check(lib.demag_energy_tucker_fp64(plan.ptr, r,
                                        _ptr(core, 3 * int(ranks[0]) * int(ranks[1]) * int(ranks[2]), f64, "core"),
                                        _ptr(V, 3 * tot, f64, "V"), _ptr(energy, 1, f64, "energy"),
                                        _stream(stream)), plan.ptr)


def demag_energy_tt(plan: Plan, ranks, G1, G2, G3, out_w, oG1, oG2, oG3, energy, stream=None):
    """Energy of a TT magnetization from its demag_apply_tt output (energy: device float64)."""
    import torch
    r1, r2 = int(ranks[0]), int(ranks[1])
    rr = (_i * 2)(r1, r2)
    f32 = torch.float32
    s1, s2, s3 = r1 * plan.n[0], r1 * r2 * plan.n[1], r2 * plan.n[2]
    M = plan.M
    _check(lib.demag_energy_tt(plan.ptr, rr, _ptr(G1, 3 * s1, f32, "G1"), _ptr(G2, 3 * s2, f32, "G2"),
                               _ptr(G3, 3 * s3, f32, "G3"), _ptr(out_w, 3 * M, f32, "out_w"),
                               _ptr(oG1, 3 * M * s1, f32, "oG1"), _ptr(oG2, 3 * M * s2, f32, "oG2"),
                               _ptr(oG3, 3 * M * s3, f32, "oG3"), _ptr(energy, 1, torch.float64, "energy"),
                               _stream(stream)), plan.ptr)


def demag_energy_tucker_phi(plan: Plan, ranks, core, V, rho, phi_core, phi_U, energy, stream=None):
    """Energy of a Tucker magnetization with phi one Tucker tensor [[phi_core; U]] of ranks rho."""
    import torch
    r = (_i * 3)(*[int(v) for v in ranks])
    rr = (_i * 3)(*[int(v) for v in rho])
    tot = sum(int(ranks[p]) * plan.n[p] for p in range(3))
    f32 = torch.float32
    _check(lib.demag_energy_tucker_phi(plan.ptr, r,
                                       _ptr(core, 3 * int(ranks[0]) * int(ranks[1]) * int(ranks[2]), f32, "core"),
                                       _ptr(V, 3 * tot, f32, "V"), rr,
                                       _ptr(phi_core, int(rho[0]) * int(rho[1]) * int(rho[2]), f32, "phi_core"),
                                       _ptr(phi_U, sum(int(rho[p]) * plan.n[p] for p in range(3)), f32, "phi_U"),
                                       _ptr(energy, 1, torch.float64, "energy"), _stream(stream)), plan.ptr)


def demag_stray_field_exact(plan: Plan, m, hd, precision="fp32", stream=None):
    """hd = -grad phi from the analytic derivative factors (no finite differences)."""
    import torch
    _check(lib.demag_stray_field_exact(plan.ptr, _ptr(m, 3 * plan.N, torch.float32, "m"),
                                       _ptr(hd, 3 * plan.N, torch.float32, "hd"), _prec(precision),
                                       _stream(stream)), plan.ptr)


def demag_sync_status(plan: Plan, stream=None):
    _check(lib.demag_sync_status(plan.ptr, _stream(stream)), plan.ptr)


def demag_set_wait_limit(plan: Plan, seconds: float):
    _check(lib.demag_set_wait_limit(plan.ptr, float(seconds)), plan.ptr)


def demag_set_fused(plan: Plan, enable: bool):
    _check(lib.demag_set_fused(plan.ptr, 1 if enable else 0), plan.ptr)


def demag_forward_schedule(plan: Plan, precision="bf16x3") -> int:
    """1 fused, 0 three-stage chain, -1 no tensor-core state for `precision` yet."""
    return lib.demag_forward_schedule(plan.ptr, _prec(precision))


def demag_autotune(plan: Plan, enable: bool = True):
    _check(lib.demag_autotune(plan.ptr, int(bool(enable))), plan.ptr)


def demag_autotune_count(plan: Plan) -> int:
    return lib.demag_autotune_count(plan.ptr)


TUNE_KINDS = {0: "fft_node_group", 1: "bf16x3_tile_width", 2: "tf32x3_tile_width", 3: "bf16x3_stages",
              4: "tf32x3_stages", 5: "bf16x3_tile_order", 6: "tf32x3_tile_order", 7: "bf16x3_store_boxes",
              8: "tf32x3_store_boxes", 9: "bf16x3_schedule"}


def demag_autotune_entry(plan: Plan, i: int) -> dict:
    kind, value = _i(), _i()
    key = (_i * 3)()
    ms, ms_default = ctypes.c_float(), ctypes.c_float()
    _check(lib.demag_autotune_entry(plan.ptr, int(i), ctypes.byref(kind), key, ctypes.byref(value),
                                    ctypes.byref(ms), ctypes.byref(ms_default)), plan.ptr)
    return {"kind": TUNE_KINDS.get(kind.value, kind.value), "key": list(key), "value": value.value,
            "ms": ms.value, "ms_default": ms_default.value}


def demag_autotune_save(plan: Plan, path: str):
    _check(lib.demag_autotune_save(plan.ptr, os.fsencode(path)), plan.ptr)


def demag_autotune_load(plan: Plan, path: str) -> int:
    n = _i()
    _check(lib.demag_autotune_load(plan.ptr, os.fsencode(path), ctypes.byref(n)), plan.ptr)
    return n.value


def demag_launch_count(plan: Plan) -> int:
    return int(lib.demag_launch_count(plan.ptr))


def demag_profile(plan: Plan, enable: bool):
    _check(lib.demag_profile(plan.ptr, 1 if enable else 0), plan.ptr)


def demag_profile_read(plan: Plan, family) -> tuple:
    """(total milliseconds, launches) recorded for a kernel family (name or id)."""
    fam = FAMILIES[family] if isinstance(family, str) else int(family)
    ms, cnt = ctypes.c_double(), ctypes.c_longlong()
    _check(lib.demag_profile_read(plan.ptr, fam, ctypes.byref(ms), ctypes.byref(cnt)), plan.ptr)
    return ms.value, cnt.value


def demag_profile_count(plan: Plan) -> int:
    return lib.demag_profile_count(plan.ptr)


_FAMILY_NAMES = {v: k for k, v in FAMILIES.items()}


def demag_profile_launch(plan: Plan, i: int) -> tuple:
    """(family name, milliseconds) of recorded launch i, in launch order."""
    fam, ms = _i(), ctypes.c_double()
    _check(lib.demag_profile_launch(plan.ptr, int(i), ctypes.byref(fam), ctypes.byref(ms)), plan.ptr)
    return _FAMILY_NAMES.get(fam.value, fam.value), ms.value


def demag_apply_full_noalloc(n, h, R: int, m, phi, c0: float = 2.15, stream=None):
    """FP32 full-format application that allocates no device memory.

    For callers that cannot allocate (a host framework's memory pool owns the
    GPU, allocations would synchronise a latency-critical loop, or plugin rules
    forbid them): the library uses a fixed 32 MiB device array of its own, and
    grids that do not fit are rejected with DemagError (DEMAG_EUNSUPPORTED).
    """
    import torch
    N = int(n[0]) * int(n[1]) * int(n[2])
    d = GridDesc((ctypes.c_int * 3)(*[int(v) for v in n]), (ctypes.c_double * 3)(*[float(v) for v in h]), int(R), float(c0))
    _check(lib.demag_apply_full_noalloc(ctypes.byref(d), _ptr(m, 3 * N, torch.float32, "m"),
                                        _ptr(phi, N, torch.float32, "phi"), _stream(stream)))
