"""Python binding of libpump (include/pump.h): argument marshalling only.

Every step of the planner runs in the library's CUDA kernels; this module
converts numpy arrays / torch tensors to pointers, passes torch's current CUDA
stream, and routes the library's device allocations to torch's caching
allocator.  It raises if the compiled library is missing; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional

import numpy as np

from . import build as _build

# status codes
OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_CAPACITY, ERR_TIMEOUT, ERR_INFEASIBLE = range(7)
NO_EARLY_STOP, EXPLORE_ONLY, STEPWISE, EXPLORE_GRID, NO_WAIT = 1, 2, 4, 8, 16
GRAPH_HSMC, GRAPH_SEPARATE_MASKS = 1, 2

EXPORT = {
    "counts": 0, "node_valid": 1, "row_ptr": 2, "col": 3, "ecost": 4, "tau": 5, "h": 6, "phi": 7, "L": 8,
    "nominal": 9, "linf": 10, "masks": 11, "plan_head": 12, "plan_parent": 13, "plan_cost": 14, "plan_mask": 15,
    "plan_popc": 16, "plan_created": 17, "plan_expanded": 18, "goal_plans": 19, "edge_box": 20, "nominal_vel": 21,
    "edge_order": 22,
}


class Aabb(C.Structure):
    _fields_ = [("lo", C.c_float * 3), ("hi", C.c_float * 3)]


class GraphParams(C.Structure):
    _fields_ = [("radius", C.c_float), ("n_particles", C.c_int32), ("n_waypoints", C.c_int32),
                ("sigma", C.c_float), ("flags", C.c_int32)]


class PlanParams(C.Structure):
    _fields_ = [("alpha", C.c_float), ("eta", C.c_float), ("lambda_", C.c_float), ("n_mc", C.c_int32),
                ("mc_substeps", C.c_int32), ("mc_seed", C.c_uint64), ("max_plans", C.c_int64),
                ("max_iterations", C.c_int32), ("flags", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("states", C.c_void_p), ("n", C.c_int32), ("start_idx", C.c_int32), ("goal_idx", C.c_void_p),
                ("n_goal", C.c_int32), ("boxes", C.c_void_p), ("n_boxes", C.c_int32), ("xi", C.c_void_p),
                ("graph", GraphParams), ("plan", PlanParams)]


class BatchConfig(C.Structure):
    _fields_ = [("cluster_size", C.c_int32), ("mbest_global", C.c_int32), ("max_clusters", C.c_int32),
                ("mask_pairs", C.c_int32), ("mask_chunk", C.c_int32), ("mask_span", C.c_int32)]


class PlanResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("chosen_plan", C.c_int32), ("cost", C.c_float), ("popc", C.c_int32),
                ("cp_hat", C.c_float), ("cp_mc", C.c_double), ("mc_collisions", C.c_int64),
                ("n_candidates", C.c_int64), ("n_kept", C.c_int64), ("n_plans", C.c_int64),
                ("n_iterations", C.c_int32), ("n_groups", C.c_int32), ("n_goal", C.c_int32),
                ("n_certified", C.c_int32), ("path_len", C.c_int32), ("path_truncated", C.c_int32),
                ("ms_masks", C.c_float), ("ms_explore", C.c_float), ("ms_select", C.c_float),
                ("fused", C.c_int32)]

    def as_dict(self) -> Dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PumpError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_str(status)} ({status})")
        self.status = status


_lib = None
_ALLOC_T = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_T = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
_hooks = []


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libpump.so from the package's build folder; raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libpump is not built ({path}); run python -m paper_1607_06886_gb300.build")
        _build.build()
    L = C.CDLL(path)
    P, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
    L.pump_set_allocator.argtypes = [_ALLOC_T, _FREE_T, P]
    L.pump_build_graph.argtypes = [P, i32, i32, P, i32, P, i32, P, C.POINTER(GraphParams), P, C.POINTER(P)]
    L.pump_graph_from_csr.argtypes = [i32, P, P, P, P, i32, i32, P, i32, P, C.POINTER(P)]
    L.pump_edge_masks.argtypes = [P, P]
    L.pump_edge_masks_list.argtypes = [P, P, C.c_int64, P, P, P]
    L.pump_explore.argtypes = [P, C.POINTER(PlanParams), f32, C.POINTER(PlanResult), P]
    L.pump_plan.argtypes = [P, C.POINTER(PlanParams), P, i32, C.POINTER(PlanResult), P]
    L.pump_plan_collect.argtypes = [P, C.POINTER(PlanResult), P]
    L.pump_certify.argtypes = [P, P, i32, i32, i32, C.c_uint64, C.POINTER(i64), C.POINTER(C.c_double), P]
    L.pump_export.argtypes = [P, i32, P, C.c_size_t, C.POINTER(C.c_size_t)]
    L.pump_graph_destroy.argtypes = [P]
    L.pump_graph_destroy.restype = None
    L.pump_explore_noalloc.argtypes = [i32, P, P, P, P, i32, i32, P, f32, C.POINTER(PlanParams), i64,
                                       P, P, P, P, P, P, P, P, C.POINTER(PlanResult), P]
    L.pump_plan_batch.argtypes = [P, i32, P, C.POINTER(BatchConfig), P, P]
    L.pump_server_create.argtypes = [i32, i64, C.POINTER(P)]
    L.pump_server_submit.argtypes = [P, C.POINTER(Request), C.POINTER(i64)]
    L.pump_server_wait.argtypes = [P, i64, C.c_double, C.POINTER(PlanResult), P, i32, C.POINTER(C.c_double)]
    L.pump_server_stats.argtypes = [P, P]
    L.pump_server_destroy.argtypes = [P]
    L.pump_server_destroy.restype = None
    L.pump_mlp_create.argtypes = [i32, P, C.c_uint64, C.POINTER(P)]
    L.pump_mlp_param_count.argtypes = [P]
    L.pump_mlp_param_count.restype = i64
    L.pump_mlp_set_params.argtypes = [P, P, i64]
    L.pump_mlp_get_params.argtypes = [P, P, i64, C.POINTER(i64)]
    L.pump_mlp_forward.argtypes = [P, P, i32, P, P]
    L.pump_mlp_gradients.argtypes = [P, P, i32, P, P, i64, P]
    L.pump_mlp_train_step.argtypes = [P, P, i32, P, P, i32, f32, f32, C.POINTER(f32), P]
    L.pump_mlp_set_data.argtypes = [P, P, i32, i32, P, P, i32]
    L.pump_mlp_set_loss.argtypes = [P, i32, i32]
    L.pump_mlp_train.argtypes = [P, i32, i32, f32, f32, C.c_uint64, P, P]
    L.pump_mlp_assemble.argtypes = [P, i32, i64, C.c_uint64, P, P]
    L.pump_mlp_propose.argtypes = [P, P, i32, i32, C.c_uint64, f32, P, P]
    L.pump_mlp_destroy.argtypes = [P]
    L.pump_mlp_destroy.restype = None
    L.pump_kernel_launches.argtypes = []
    L.pump_kernel_launches.restype = C.c_uint64
    L.pump_status_str.argtypes = [C.c_int]
    L.pump_status_str.restype = C.c_char_p
    _lib = L
    return L


def plan_batch(graphs, params, config: Optional["BatchConfig"] = None, stream: Optional[int] = None):
    """pump_plan_batch: one query per graph (params: one PlanParams, or one per graph).  Returns
    (rc, list of result dicts)."""
    graphs = list(graphs)
    nq = len(graphs)
    if isinstance(params, PlanParams):
        params = [params] * nq
    if len(params) != nq:
        raise ValueError("one PlanParams per graph")
    handles = (C.c_void_p * nq)(*[g._h for g in graphs])
    prm = (PlanParams * nq)(*params)
    res = (PlanResult * nq)()
    rc = load().pump_plan_batch(C.cast(handles, C.c_void_p), nq, C.cast(prm, C.c_void_p),
                                C.byref(config) if config is not None else None, C.cast(res, C.c_void_p),
                                current_stream() if stream is None else stream)
    out = []
    for r in res:
        d = r.as_dict()
        d["rc"] = r.status
        out.append(d)
    return rc, out


class Server:
    """pump_server: continuous batching over `slots` CUDA streams within `device_bytes` (estimated)."""

    def __init__(self, slots: int, device_bytes: int):
        h = C.c_void_p()
        rc = load().pump_server_create(int(slots), int(device_bytes), C.byref(h))
        if rc:
            raise PumpError(rc, "pump_server_create")
        self._h = h

    def submit(self, states, goal_idx, boxes, xi, radius: float, n_particles: int, n_waypoints: int, sigma: float,
               plan: "PlanParams", start_idx: int = 0) -> int:
        # host arrays (the server copies them before submit returns)
        st = np.ascontiguousarray(states, dtype=np.float32).reshape(-1, 6)
        gi = np.ascontiguousarray(goal_idx, dtype=np.int32).ravel()
        bx = np.ascontiguousarray(boxes, dtype=np.float32).reshape(-1, 6)
        x = np.ascontiguousarray(xi, dtype=np.float32)
        req = Request(st.ctypes.data, st.shape[0], int(start_idx), gi.ctypes.data, gi.size,
                      bx.ctypes.data if bx.size else None, bx.shape[0], x.ctypes.data,
                      GraphParams(float(radius), int(n_particles), int(n_waypoints), float(sigma), 0), plan)
        t = C.c_int64()
        rc = load().pump_server_submit(self._h, C.byref(req), C.byref(t))
        if rc:
            raise PumpError(rc, "pump_server_submit")
        return int(t.value)

    def wait(self, ticket: int, timeout: float = 600.0, path_cap: int = 4097) -> Dict:
        res = PlanResult()
        path = np.zeros(max(path_cap, 1), np.int32)
        lat = C.c_double()
        rc = load().pump_server_wait(self._h, int(ticket), float(timeout), C.byref(res), _ptr(path), int(path_cap),
                                     C.byref(lat))
        d = res.as_dict()
        d["rc"] = rc
        d["path"] = path[:max(min(res.path_len, path_cap), 0)].copy()
        d["latency_ms"] = float(lat.value)
        return d

    def stats(self) -> Dict:
        c = np.zeros(8, np.int64)
        load().pump_server_stats(self._h, _ptr(c))
        keys = ("submitted", "admitted", "completed", "queued", "running", "peak_running", "bytes_in_use", "peak_bytes")
        return {k: int(v) for k, v in zip(keys, c)}

    def close(self):
        if self._h:
            load().pump_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The learned sampling proposal's network (pump_mlp_*): BF16 tensor-core products, FP32
    master weights, Adam, and a device-side training loop replayed as a CUDA graph."""

    def __init__(self, dims, seed: int = 0):
        self.dims = [int(d) for d in dims]
        d = np.asarray(self.dims, np.int32)
        h = C.c_void_p()
        rc = load().pump_mlp_create(len(self.dims) - 1, d.ctypes.data, int(seed), C.byref(h))
        if rc:
            raise PumpError(rc, "pump_mlp_create")
        self._h = h
        self.n_params = int(load().pump_mlp_param_count(h))

    def _check(self, rc, what):
        if rc:
            raise PumpError(rc, what)

    def set_params(self, params) -> None:
        p = np.ascontiguousarray(params, np.float32)
        self._check(load().pump_mlp_set_params(self._h, p.ctypes.data, p.size), "pump_mlp_set_params")

    def get_params(self):
        p = np.zeros(self.n_params, np.float32)
        steps = C.c_int64()
        self._check(load().pump_mlp_get_params(self._h, p.ctypes.data, p.size, C.byref(steps)), "pump_mlp_get_params")
        return p, int(steps.value)

    def forward(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, np.float32)
        y = np.zeros((x.shape[0], self.dims[-1]), np.float32)
        self._check(load().pump_mlp_forward(self._h, x.ctypes.data, x.shape[0], y.ctypes.data, current_stream()),
                    "pump_mlp_forward")
        return y

    def gradients(self, x, dy) -> np.ndarray:
        x = np.ascontiguousarray(x, np.float32)
        dy = np.ascontiguousarray(dy, np.float32)
        g = np.zeros(self.n_params, np.float32)
        self._check(load().pump_mlp_gradients(self._h, x.ctypes.data, x.shape[0], dy.ctypes.data, g.ctypes.data,
                                              g.size, current_stream()), "pump_mlp_gradients")
        return g

    def train_step(self, x, targets, n_targets, lr: float, vmax: float) -> float:
        x = np.ascontiguousarray(x, np.float32)
        t = np.ascontiguousarray(targets, np.float32)
        n = np.ascontiguousarray(n_targets, np.int32)
        loss = C.c_float()
        self._check(load().pump_mlp_train_step(self._h, x.ctypes.data, x.shape[0], t.ctypes.data, n.ctypes.data,
                                               t.shape[1], float(lr), float(vmax), C.byref(loss), current_stream()),
                    "pump_mlp_train_step")
        return float(loss.value)

    def set_loss(self, kind: int, latent_col: int = 0) -> None:
        """0: winner takes all over the targets; 1: path-indexed by Phi(x[latent_col])."""
        self._check(load().pump_mlp_set_loss(self._h, int(kind), int(latent_col)), "pump_mlp_set_loss")

    def set_data(self, feat, targets, n_targets) -> None:
        f = np.ascontiguousarray(feat, np.float32)
        t = np.ascontiguousarray(targets, np.float32)
        n = np.ascontiguousarray(n_targets, np.int32)
        self._check(load().pump_mlp_set_data(self._h, f.ctypes.data, f.shape[1], f.shape[0], t.ctypes.data,
                                             n.ctypes.data, t.shape[1]), "pump_mlp_set_data")

    def train(self, batch: int, steps: int, lr: float, vmax: float, seed: int) -> np.ndarray:
        tr = np.zeros(max(int(steps), 1), np.float32)
        self._check(load().pump_mlp_train(self._h, int(batch), int(steps), float(lr), float(vmax), int(seed),
                                          tr.ctypes.data, current_stream()), "pump_mlp_train")
        return tr[:int(steps)]

    def assemble(self, batch: int, t: int, seed: int):
        x = np.zeros((batch, self.dims[0]), np.float32)
        env = np.zeros(batch, np.int32)
        self._check(load().pump_mlp_assemble(self._h, int(batch), int(t), int(seed), x.ctypes.data, env.ctypes.data),
                    "pump_mlp_assemble")
        return x, env

    def propose(self, feat, count: int, seed: int, vmax: float) -> np.ndarray:
        f = np.ascontiguousarray(feat, np.float32).ravel()
        out = np.zeros((int(count), 6), np.float32)
        self._check(load().pump_mlp_propose(self._h, f.ctypes.data, f.size, int(count), int(seed), float(vmax),
                                            out.ctypes.data, current_stream()), "pump_mlp_propose")
        return out

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().pump_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches() -> int:
    return int(load().pump_kernel_launches())


def status_str(st: int) -> str:
    return load().pump_status_str(int(st)).decode()


def use_torch_allocator() -> None:
    """Route the library's device allocations to torch's caching allocator.

    Each block is allocated on the stream the library will use it on (the caching allocator then
    reuses a freed block only in that stream's order), on the calling thread's current device."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                          int(stream) if stream else 0))
        except Exception:  # allocation failure is reported to the library as NULL
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC_T(_alloc), _FREE_T(_free)
    _hooks[:] = [a, f]
    load().pump_set_allocator(a, f, None)


def current_stream() -> Optional[int]:
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def _ptr(a) -> Optional[int]:
    """Pointer of a numpy array (host) or torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return int(a.data_ptr())
    return int(a.ctypes.data)


def _np(a, dtype):
    if hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


def explore_noalloc(n: int, row_ptr, col, ecost, emask, n_particles: int, start_idx: int, is_goal, radius: float,
                    params: PlanParams, capacity: int, out: Dict, stream: Optional[int] = None) -> Dict:
    """pump_explore_noalloc on caller-owned device tensors (inputs and the `out` arena buffers:
    plan_head, plan_parent, plan_cost, plan_mask, plan_popc, plan_created, plan_expanded, goal_plans)."""
    res = PlanResult()
    rc = load().pump_explore_noalloc(int(n), _ptr(row_ptr), _ptr(col), _ptr(ecost), _ptr(emask), int(n_particles),
                                     int(start_idx), _ptr(is_goal), float(radius), C.byref(params), int(capacity),
                                     _ptr(out["plan_head"]), _ptr(out["plan_parent"]), _ptr(out["plan_cost"]),
                                     _ptr(out["plan_mask"]), _ptr(out["plan_popc"]), _ptr(out["plan_created"]),
                                     _ptr(out["plan_expanded"]), _ptr(out["goal_plans"]), C.byref(res),
                                     current_stream() if stream is None else stream)
    d = res.as_dict()
    d["rc"] = rc
    return d


def default_plan_params(alpha=0.01, eta=2.0, lam=0.5, n_mc=10000, mc_substeps=4, mc_seed=0,
                        max_plans=1 << 22, max_iterations=1 << 20, flags=0) -> PlanParams:
    return PlanParams(alpha, eta, lam, n_mc, mc_substeps, mc_seed, max_plans, max_iterations, flags)


class Graph:
    """A device-resident planning graph (pump_graph)."""

    def __init__(self, handle: int, keep=()):
        self._h = C.c_void_p(handle)
        self._keep = keep

    @classmethod
    def build(cls, states, goal_idx, boxes, xi, radius: float, n_particles: int, n_waypoints: int,
              sigma: float, start_idx: int = 0, stream: Optional[int] = None, flags: int = 0) -> "Graph":
        """pump_build_graph; flags: GRAPH_HSMC for Half-Space Monte Carlo masks, GRAPH_SEPARATE_MASKS
        to keep the masks of every query in their own launch."""
        L = load()
        st = _np(states, np.float32)
        gi = _np(goal_idx, np.int32)
        bx = _np(boxes, np.float32)
        x = _np(xi, np.float32)
        n = int(st.shape[0])
        nb = int(bx.shape[0]) if bx is not None else 0
        prm = GraphParams(float(radius), int(n_particles), int(n_waypoints), float(sigma), int(flags))
        out = C.c_void_p()
        s = current_stream() if stream is None else stream
        rc = L.pump_build_graph(_ptr(st), n, int(start_idx), _ptr(gi), int(len(gi)), _ptr(bx) if nb else None, nb,
                                _ptr(x), C.byref(prm), s, C.byref(out))
        if rc:
            raise PumpError(rc, "pump_build_graph")
        return cls(out.value)

    @classmethod
    def from_csr(cls, n: int, row_ptr, col, ecost, emask, n_particles: int, start_idx: int, goal_idx,
                 stream: Optional[int] = None) -> "Graph":
        L = load()
        rp = _np(row_ptr, np.int32); cl = _np(col, np.int32); ec = _np(ecost, np.float32)
        em = _np(emask, np.uint32); gi = _np(goal_idx, np.int32)
        out = C.c_void_p()
        s = current_stream() if stream is None else stream
        rc = L.pump_graph_from_csr(int(n), _ptr(rp), _ptr(cl), _ptr(ec), _ptr(em), int(n_particles), int(start_idx),
                                   _ptr(gi), int(len(gi)), s, C.byref(out))
        if rc:
            raise PumpError(rc, "pump_graph_from_csr")
        return cls(out.value)

    def close(self):
        if self._h and self._h.value:
            load().pump_graph_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def edge_masks(self, stream: Optional[int] = None):
        rc = load().pump_edge_masks(self._h, current_stream() if stream is None else stream)
        if rc:
            raise PumpError(rc, "pump_edge_masks")

    def edge_masks_list(self, edges_ptr: int, n: int, out_ptr: int, bad_ptr: int = 0,
                        stream: Optional[int] = None) -> int:
        """pump_edge_masks_list on device buffers (int32 edge ids, n x N/32 uint32 rows, optional uint32
        count of bad ids); returns the status."""
        return load().pump_edge_masks_list(self._h, C.c_void_p(edges_ptr), int(n), C.c_void_p(out_ptr),
                                           C.c_void_p(bad_ptr or None), current_stream() if stream is None else stream)

    def explore(self, params: PlanParams, radius: float = 0.0, stream: Optional[int] = None) -> Dict:
        res = PlanResult()
        rc = load().pump_explore(self._h, C.byref(params), float(radius), C.byref(res),
                                 current_stream() if stream is None else stream)
        d = res.as_dict()
        d["rc"] = rc
        return d

    def plan(self, params: PlanParams, path_cap: int = 4096, stream: Optional[int] = None) -> Dict:
        res = PlanResult()
        path = np.zeros(max(path_cap, 1), np.int32)
        rc = load().pump_plan(self._h, C.byref(params), _ptr(path), int(path_cap), C.byref(res),
                              current_stream() if stream is None else stream)
        d = res.as_dict()
        d["rc"] = rc
        d["path"] = path[:res.path_len].copy()
        return d

    def collect(self, stream: Optional[int] = None) -> Dict:
        """pump_plan_collect: wait for the stream and read the last query's Explore counters (for
        queries enqueued with NO_WAIT)."""
        res = PlanResult()
        rc = load().pump_plan_collect(self._h, C.byref(res), current_stream() if stream is None else stream)
        d = res.as_dict()
        d["rc"] = rc
        return d

    def certify(self, path, n_mc: int, substeps: int, seed: int, stream: Optional[int] = None):
        p = _np(path, np.int32)
        n = C.c_int64()
        cp = C.c_double()
        rc = load().pump_certify(self._h, _ptr(p), int(len(p)), int(n_mc), int(substeps), C.c_uint64(seed),
                                 C.byref(n), C.byref(cp), current_stream() if stream is None else stream)
        if rc:
            raise PumpError(rc, "pump_certify")
        return int(n.value), float(cp.value)

    def export(self, what: str) -> np.ndarray:
        L = load()
        code = EXPORT[what]
        need = C.c_size_t()
        rc = L.pump_export(self._h, code, None, 0, C.byref(need))
        if rc and need.value == 0:
            raise PumpError(rc, f"pump_export({what})")
        buf = np.zeros(max(int(need.value), 1), np.uint8)
        rc = L.pump_export(self._h, code, _ptr(buf), int(need.value), C.byref(need))
        if rc:
            raise PumpError(rc, f"pump_export({what})")
        raw = buf[:int(need.value)]
        cnt = self.counts() if what != "counts" else None
        if what == "counts":
            return raw.view(np.int64)
        n, E, P, G, N, W, w = (int(cnt[k]) for k in range(7))
        shapes = {"node_valid": (np.uint8, (n,)), "row_ptr": (np.int32, (n + 1,)), "col": (np.int32, (E,)),
                  "ecost": (np.float32, (E,)), "tau": (np.float32, (E,)), "h": (np.float32, (E,)),
                  "phi": (np.float32, (E, 4)), "L": (np.float32, (E, 3)), "nominal": (np.float32, (E, W, 3)),
                  "linf": (np.float32, (3,)), "masks": (np.uint32, (E, w)), "plan_head": (np.int32, (P,)),
                  "plan_parent": (np.int32, (P,)), "plan_cost": (np.float32, (P,)), "plan_mask": (np.uint32, (P, w)),
                  "plan_popc": (np.int32, (P,)), "plan_created": (np.int32, (P,)),
                  "plan_expanded": (np.int32, (P,)), "goal_plans": (np.int32, (G,)),
                  "edge_box": (np.float32, (E, 6)), "nominal_vel": (np.float32, (E, W, 3)),
                  "edge_order": (np.int32, (E, 2))}
        dt, shp = shapes[what]
        return raw.view(dt).reshape(shp).copy()

    def counts(self) -> np.ndarray:
        L = load()
        buf = np.zeros(8, np.int64)
        need = C.c_size_t()
        rc = L.pump_export(self._h, EXPORT["counts"], _ptr(buf), 64, C.byref(need))
        if rc:
            raise PumpError(rc, "pump_export(counts)")
        return buf
