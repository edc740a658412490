"""ctypes binding of libdagexec (include/dagexec.h): same names, argument
marshalling only.  Every computation runs in the library's CUDA kernels; there
is no Python or CPU fallback: if the compiled library is missing, importing
this module's functions raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libdagexec.so")

i32, u32, u64, f32 = C.c_int32, C.c_uint32, C.c_uint64, C.c_float

# dag_status
DAG_OK, DAG_EINVAL, DAG_ECYCLE, DAG_ESHAPE, DAG_EDTYPE, DAG_EMULTIWRITER, DAG_ENOMEM, DAG_EBUSY, \
    DAG_ETIMEOUT, DAG_EDEVICE, DAG_EUNSUPPORTED = range(11)
STATUS_NAMES = {0: "DAG_OK", 1: "DAG_EINVAL", 2: "DAG_ECYCLE", 3: "DAG_ESHAPE", 4: "DAG_EDTYPE",
                5: "DAG_EMULTIWRITER", 6: "DAG_ENOMEM", 7: "DAG_EBUSY", 8: "DAG_ETIMEOUT", 9: "DAG_EDEVICE",
                10: "DAG_EUNSUPPORTED"}
DAG_F32, DAG_BF16 = 0, 1
DAG_OP_GEMM, DAG_OP_ADD, DAG_OP_SOFTMAX, DAG_OP_UNARY = 0, 1, 2, 3
DAG_ACT_NONE, DAG_ACT_RELU, DAG_ACT_GELU = 0, 1, 2
DAG_BUF_INPUT, DAG_BUF_OUTPUT, DAG_BUF_RESIDENT = 1, 2, 4
DAG_SCHED_RANK_MODEL, DAG_SCHED_RANK_GIVEN, DAG_SCHED_FIFO = 0, 1, 2
DAG_F32_GEMM_TENSOR, DAG_F32_GEMM_SIMT, DAG_F32_GEMM_TENSOR_NARROW, DAG_F32_GEMM_TENSOR_WIDE = 0, 1, 2, 3
DAG_RANK_UPWARD, DAG_RANK_CRITICAL_PATH = 0, 1
DAG_FUSE_NONE, DAG_FUSE_ACT, DAG_FUSE_ALL = 0, 1, 2
DAG_TC_GIVEN, DAG_TC_WHOLE, DAG_TC_PER_KERNEL = 0, 1, 2


class dag_buffer_desc(C.Structure):
    _fields_ = [("rows", i32), ("cols", i32), ("dtype", i32), ("flags", u32), ("view_of", i32),
                ("col_offset", i32)]


class dag_node_desc(C.Structure):
    _fields_ = [("op", i32), ("a", i32), ("b", i32), ("bias", i32), ("out", i32), ("trans_b", i32),
                ("act", i32), ("scale", f32), ("batch", i32), ("component", i32)]


class dag_edge(C.Structure):
    _fields_ = [("src_node", i32), ("src_buf", i32), ("dst_node", i32), ("dst_buf", i32)]


class dag_options(C.Structure):
    _fields_ = [("timeout_ns", u64), ("trace", i32), ("max_ctas", i32), ("scheduler", i32),
                ("tile_override", i32), ("node_cost_us", C.POINTER(f32)), ("debug_never_ready", i32),
                ("use_graph", i32), ("autotune", i32), ("f32_gemm", i32), ("split_k", i32), ("fuse", i32),
                ("keep_layout", i32), ("rank_form", i32), ("merge", i32)]


class dag_cq_options(C.Structure):
    _fields_ = [("n_queues", i32), ("components", i32), ("fifo", i32), ("pad", i32), ("timeout_ns", u64),
                ("node_start_us", C.POINTER(f32)), ("node_end_us", C.POINTER(f32)),
                ("node_queue", C.POINTER(i32))]


class dag_cq_result(C.Structure):
    _fields_ = [("device_us", C.c_double), ("host_us", C.c_double), ("gap_us", C.c_double),
                ("n_components", i32), ("n_callbacks", i32)]


class dag_copy_class(C.Structure):
    _fields_ = [("node", i32), ("buf", i32), ("is_write", i32), ("isolated", i32)]


class dag_edge_class(C.Structure):
    _fields_ = [("src_node", i32), ("src_buf", i32), ("dst_node", i32), ("dst_buf", i32), ("inter", i32)]


class dag_analysis(C.Structure):
    _fields_ = [("n_nodes", i32), ("cls", C.POINTER(i32)), ("topo", C.POINTER(i32)),
                ("copies", C.POINTER(dag_copy_class)), ("cap_copies", i32), ("n_copies", i32),
                ("edge_cls", C.POINTER(dag_edge_class)), ("cap_edges", i32), ("n_edge_cls", i32)]


class dag_trace_record(C.Structure):
    _fields_ = [("node", i32), ("r0", i32), ("r1", i32), ("c0", i32), ("c1", i32), ("start_ticket", u32),
                ("end_ticket", u32), ("smid", u32), ("split", i32), ("pad", i32), ("t_claim_ns", u64),
                ("t_start_ns", u64), ("t_work_ns", u64), ("t_end_ns", u64)]


class dag_plan_info(C.Structure):
    _fields_ = [("n_tiles", i32), ("n_counters", i32), ("n_waits", i32), ("grid", i32), ("smem_bytes", i32),
                ("flops", C.c_double), ("bytes", C.c_double), ("critical_path_us", C.c_double),
                ("work_bound_us", C.c_double), ("tile_override", i32), ("scheduler", i32), ("tuned_us", C.c_double),
                ("buffer_bytes", C.c_double)]


class dag_batch_item(C.Structure):
    _fields_ = [("nodes", C.POINTER(dag_node_desc)), ("n_nodes", i32), ("buffers", C.POINTER(dag_buffer_desc)),
                ("n_buffers", i32)]


class dag_model_desc(C.Structure):
    _fields_ = [("nodes", C.POINTER(dag_node_desc)), ("n_nodes", i32), ("buffers", C.POINTER(dag_buffer_desc)),
                ("n_buffers", i32), ("weights", C.POINTER(C.c_void_p)), ("node_cost_us", C.POINTER(f32))]


class dag_request_info(C.Structure):
    _fields_ = [("model", i32), ("status", i32), ("t_arrive_s", C.c_double), ("t_launch_s", C.c_double),
                ("t_done_s", C.c_double)]


class DagError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


_lib = None
_lock = threading.Lock()

_SIGS = {
    "dag_create": (i32, [C.POINTER(dag_node_desc), C.c_int, C.POINTER(dag_edge), C.c_int,
                         C.POINTER(dag_buffer_desc), C.c_int, C.POINTER(dag_options), C.POINTER(C.c_void_p)]),
    "dag_batch_create": (i32, [C.POINTER(dag_batch_item), C.c_int, C.POINTER(dag_options), C.POINTER(C.c_void_p)]),
    "dag_set_input": (i32, [C.c_void_p, C.c_int, C.c_void_p]),
    "dag_set_output": (i32, [C.c_void_p, C.c_int, C.c_void_p]),
    "dag_submit": (i32, [C.c_void_p, C.c_void_p]),
    "dag_submit_coarse": (i32, [C.c_void_p, C.c_void_p]),
    "dag_submit_cq": (i32, [C.c_void_p, C.POINTER(dag_cq_options), C.POINTER(dag_cq_result)]),
    "dag_wait": (i32, [C.c_void_p, u64]),
    "dag_get_output": (i32, [C.c_void_p, C.c_int, C.c_void_p]),
    "dag_device_ptr": (C.c_void_p, [C.c_void_p, C.c_int, C.POINTER(C.c_int64)]),
    "dag_destroy": (i32, [C.c_void_p]),
    "dag_last_error": (C.c_char_p, []),
    "dag_host_alloc": (C.c_void_p, [C.c_size_t]),
    "dag_host_free": (None, [C.c_void_p]),
    "dag_analyze": (i32, [C.POINTER(dag_node_desc), C.c_int, C.POINTER(dag_edge), C.c_int,
                          C.POINTER(dag_buffer_desc), C.c_int, C.POINTER(dag_analysis)]),
    "dag_trace_get": (i32, [C.c_void_p, C.POINTER(dag_trace_record), C.c_int, C.POINTER(C.c_int)]),
    "dag_plan_get": (i32, [C.c_void_p, C.POINTER(dag_plan_info)]),
    "dag_tiles_get": (i32, [C.c_void_p, C.POINTER(i32), C.c_int, C.POINTER(C.c_int)]),
    "dag_plan_host": (i32, [C.POINTER(dag_node_desc), C.c_int, C.POINTER(dag_edge), C.c_int,
                            C.POINTER(dag_buffer_desc), C.c_int, C.POINTER(dag_options), C.c_int,
                            C.POINTER(i32), C.c_int, C.POINTER(C.c_int), C.POINTER(dag_plan_info)]),
    "dag_fusion_get": (i32, [C.c_void_p, C.POINTER(i32), C.c_int, C.POINTER(C.c_int)]),
    "dag_merge_get": (i32, [C.c_void_p, C.POINTER(i32), C.POINTER(i32), C.c_int, C.POINTER(C.c_int)]),
    "dag_merge_host": (i32, [C.POINTER(dag_node_desc), C.c_int, C.POINTER(dag_buffer_desc), C.c_int,
                             C.POINTER(dag_options), C.POINTER(i32), C.POINTER(i32)]),
    "dag_fusion_host": (i32, [C.POINTER(dag_node_desc), C.c_int, C.POINTER(dag_edge), C.c_int,
                              C.POINTER(dag_buffer_desc), C.c_int, C.POINTER(dag_options), C.POINTER(i32)]),
    "dag_set_peaks": (None, [C.c_double, C.c_double, C.c_double]),
    "dag_set_device": (i32, [C.c_int]),
    "dag_trace_stamps": (i32, [C.c_void_p, C.POINTER(u64), C.c_int, C.POINTER(C.c_int)]),
    "dag_trace_launch": (i32, [C.c_void_p, C.POINTER(u64)]),
    "dag_node_costs_get": (i32, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "dag_poll": (i32, [C.c_void_p]),
    "dag_server_create": (i32, [C.POINTER(dag_model_desc), C.c_int, C.c_int, C.c_size_t, C.POINTER(dag_options),
                                C.POINTER(C.c_void_p)]),
    "dag_server_set_io": (i32, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "dag_server_warm": (i32, [C.c_void_p, C.c_int, C.c_int]),
    "dag_server_submit": (i32, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                C.POINTER(C.c_uint64)]),
    "dag_server_progress": (C.c_int, [C.c_void_p]),
    "dag_server_wait": (i32, [C.c_void_p, C.c_uint64, C.c_uint64, C.POINTER(dag_request_info)]),
    "dag_server_simulate": (i32, [C.c_void_p, C.POINTER(i32), C.c_int, C.c_double, C.c_uint64,
                                  C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "dag_server_slots": (C.c_int, [C.c_void_p]),
    "dag_server_destroy": (i32, [C.c_void_p]),
    "dag_mlp_create": (i32, [C.c_int, C.POINTER(C.c_void_p)]),
    "dag_mlp_param_count": (C.c_int, [C.c_void_p]),
    "dag_mlp_set_params": (i32, [C.c_void_p, C.c_void_p, C.c_int]),
    "dag_mlp_get_params": (i32, [C.c_void_p, C.c_void_p, C.c_int]),
    "dag_mlp_loss_grad": (i32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_float), C.c_void_p]),
    "dag_mlp_train": (i32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_float]),
    "dag_mlp_predict": (i32, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "dag_mlp_destroy": (i32, [C.c_void_p]),
    "dag_run_noalloc": (i32, [C.POINTER(dag_node_desc), C.c_int, C.POINTER(dag_buffer_desc), C.c_int,
                              C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.POINTER(dag_options), C.c_void_p]),
}


def lib():
    """The loaded library; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libdagexec.so is not built ({LIB_PATH}); run __graft_entry__.build()")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().dag_last_error().decode(errors="replace")


def check(status: int, where: str) -> None:
    if status != DAG_OK:
        raise DagError(status, where, last_error())


# thin wrappers with the C names ------------------------------------------------
def _arr(ctype, items):
    items = list(items)
    return (ctype * max(1, len(items)))(*items), len(items)


def dag_create(nodes, edges, buffers, options: Optional[dag_options] = None) -> C.c_void_p:
    na, nn = _arr(dag_node_desc, nodes)
    ea, ne = _arr(dag_edge, edges)
    ba, nb = _arr(dag_buffer_desc, buffers)
    h = C.c_void_p()
    check(lib().dag_create(na, nn, ea, ne, ba, nb, C.byref(options) if options else None, C.byref(h)), "dag_create")
    return h


def dag_batch_create(items, options: Optional[dag_options] = None) -> C.c_void_p:
    """items: list of (nodes, buffers) lists of ABI structs."""
    keep = []
    arr = (dag_batch_item * max(1, len(items)))()
    for i, (nodes, buffers) in enumerate(items):
        na, nn = _arr(dag_node_desc, nodes)
        ba, nb = _arr(dag_buffer_desc, buffers)
        keep += [na, ba]
        arr[i] = dag_batch_item(C.cast(na, C.POINTER(dag_node_desc)), nn, C.cast(ba, C.POINTER(dag_buffer_desc)), nb)
    h = C.c_void_p()
    check(lib().dag_batch_create(arr, len(items), C.byref(options) if options else None, C.byref(h)),
          "dag_batch_create")
    return h


def dag_analyze(nodes, edges, buffers, cap: int = 4096) -> dict:
    na, nn = _arr(dag_node_desc, nodes)
    ea, ne = _arr(dag_edge, edges)
    ba, nb = _arr(dag_buffer_desc, buffers)
    cls = (i32 * max(1, nn))()
    topo = (i32 * max(1, nn))()
    copies = (dag_copy_class * cap)()
    ecls = (dag_edge_class * cap)()
    a = dag_analysis(nn, cls, topo, copies, cap, 0, ecls, cap, 0)
    check(lib().dag_analyze(na, nn, ea, ne, ba, nb, C.byref(a)), "dag_analyze")
    return {
        "cls": list(cls[:nn]), "topo": list(topo[:nn]),
        "copies": [(c.node, c.buf, c.is_write, c.isolated) for c in copies[:min(cap, a.n_copies)]],
        "edges": [(e.src_node, e.src_buf, e.dst_node, e.dst_buf, e.inter) for e in ecls[:min(cap, a.n_edge_cls)]],
    }


def dag_plan_host(nodes, edges, buffers, options: Optional[dag_options] = None, n_sm: int = 148):
    na, nn = _arr(dag_node_desc, nodes)
    ea, ne = _arr(dag_edge, edges)
    ba, nb = _arr(dag_buffer_desc, buffers)
    n = C.c_int(0)
    info = dag_plan_info()
    opt = C.byref(options) if options else None
    check(lib().dag_plan_host(na, nn, ea, ne, ba, nb, opt, n_sm, None, 0, C.byref(n), C.byref(info)), "dag_plan_host")
    out = (i32 * (6 * max(1, n.value)))()
    check(lib().dag_plan_host(na, nn, ea, ne, ba, nb, opt, n_sm, out, n.value, C.byref(n), None), "dag_plan_host")
    import numpy as np
    return np.frombuffer(out, dtype=np.int32)[: 6 * n.value].reshape(-1, 6).copy(), info


def dag_fusion_host(nodes, edges, buffers, options: Optional[dag_options] = None):
    """Per kernel: the GEMM whose epilogue computes it, or -1 (see dag_fusion_get)."""
    na, nn = _arr(dag_node_desc, nodes)
    ea, ne = _arr(dag_edge, edges)
    ba, nb = _arr(dag_buffer_desc, buffers)
    out = (i32 * max(1, nn))()
    check(lib().dag_fusion_host(na, nn, ea, ne, ba, nb, C.byref(options) if options else None, out),
          "dag_fusion_host")
    return list(out[:nn])


def dag_fusion_get(h):
    n = C.c_int(0)
    check(lib().dag_fusion_get(h, None, 0, C.byref(n)), "dag_fusion_get")
    out = (i32 * max(1, n.value))()
    check(lib().dag_fusion_get(h, out, n.value, C.byref(n)), "dag_fusion_get")
    return list(out[:n.value])


def dag_merge_get(h):
    """Per kernel: (the kernel whose tiles compute it or -1, its first column
    in that merged GEMM) (see dag_merge_get in dagexec.h)."""
    n = C.c_int(0)
    check(lib().dag_merge_get(h, None, None, 0, C.byref(n)), "dag_merge_get")
    lead, off = (i32 * max(1, n.value))(), (i32 * max(1, n.value))()
    check(lib().dag_merge_get(h, lead, off, n.value, C.byref(n)), "dag_merge_get")
    return list(lead[:n.value]), list(off[:n.value])


def dag_merge_host(nodes, buffers, options: Optional[dag_options] = None):
    """dag_merge_get without a device: the planner's merge of sibling GEMMs."""
    na, nn = _arr(dag_node_desc, nodes)
    ba, nb = _arr(dag_buffer_desc, buffers)
    lead, off = (i32 * max(1, nn))(), (i32 * max(1, nn))()
    check(lib().dag_merge_host(na, nn, ba, nb, C.byref(options) if options else None, lead, off), "dag_merge_host")
    return list(lead[:nn]), list(off[:nn])


def dag_set_input(h, buf: int, host_ptr) -> None:
    check(lib().dag_set_input(h, buf, host_ptr), "dag_set_input")


def dag_set_output(h, buf: int, host_ptr) -> None:
    check(lib().dag_set_output(h, buf, host_ptr), "dag_set_output")


def dag_submit(h, stream: int = 0) -> None:
    check(lib().dag_submit(h, C.c_void_p(stream)), "dag_submit")


def dag_submit_coarse(h, stream: int = 0) -> None:
    check(lib().dag_submit_coarse(h, C.c_void_p(stream)), "dag_submit_coarse")


def dag_submit_cq(h, n_queues: int = 1, components: int = 1, fifo: int = 0, timeout_ns: int = 0,
                  n_nodes: int = 0, queues: bool = False):
    """The paper's Alg. 1 on CUDA streams (synchronous).  Returns the result
    struct and, if n_nodes > 0, per-kernel (start_us, end_us) arrays, and with
    `queues` also the queue each kernel was sent to."""
    import numpy as np
    o = dag_cq_options(n_queues=n_queues, components=components, fifo=fifo, timeout_ns=timeout_ns)
    ts = te = qs = None
    if n_nodes:
        ts = np.zeros(n_nodes, np.float32)
        te = np.zeros(n_nodes, np.float32)
        o.node_start_us = ts.ctypes.data_as(C.POINTER(f32))
        o.node_end_us = te.ctypes.data_as(C.POINTER(f32))
        if queues:
            qs = np.full(n_nodes, -1, np.int32)
            o.node_queue = qs.ctypes.data_as(C.POINTER(i32))
    r = dag_cq_result()
    check(lib().dag_submit_cq(h, C.byref(o), C.byref(r)), "dag_submit_cq")
    return (r, ts, te, qs) if queues else (r, ts, te)


def dag_wait(h, timeout_ns: int = 30_000_000_000) -> int:
    """Returns the status (does not raise on DAG_ETIMEOUT so callers can test it)."""
    return int(lib().dag_wait(h, timeout_ns))


def dag_get_output(h, buf: int, host_ptr) -> None:
    check(lib().dag_get_output(h, buf, host_ptr), "dag_get_output")


def dag_device_ptr(h, buf: int):
    ld = C.c_int64(0)
    p = lib().dag_device_ptr(h, buf, C.byref(ld))
    return p, ld.value


def dag_destroy(h) -> None:
    check(lib().dag_destroy(h), "dag_destroy")


def dag_host_alloc(nbytes: int) -> int:
    p = lib().dag_host_alloc(nbytes)
    if not p:
        raise DagError(DAG_ENOMEM, "dag_host_alloc", last_error())
    return p


def dag_host_free(p) -> None:
    lib().dag_host_free(p)


def dag_trace_get(h):
    n = C.c_int(0)
    check(lib().dag_trace_get(h, None, 0, C.byref(n)), "dag_trace_get")
    recs = (dag_trace_record * max(1, n.value))()
    check(lib().dag_trace_get(h, recs, n.value, C.byref(n)), "dag_trace_get")
    return recs[: n.value]


def dag_trace_stamps(h):
    """(n_tiles, 10) uint64 array of per-phase %globaltimer stamps (see dagexec.h)."""
    import numpy as np
    n = C.c_int(0)
    check(lib().dag_trace_stamps(h, None, 0, C.byref(n)), "dag_trace_stamps")
    out = (u64 * (10 * max(1, n.value)))()
    check(lib().dag_trace_stamps(h, out, n.value, C.byref(n)), "dag_trace_stamps")
    return np.frombuffer(out, dtype=np.uint64)[: 10 * n.value].reshape(-1, 10).copy()


def dag_run_noalloc(nodes, buffers, buffer_ptrs, row_pitch, options: Optional[dag_options] = None,
                    stream: int = 0) -> int:
    """Run a DAG on caller-owned device buffers with no device allocation
    (synchronous); returns the status so callers can test DAG_ENOMEM etc."""
    na, nn = _arr(dag_node_desc, nodes)
    ba, nb = _arr(dag_buffer_desc, buffers)
    pa = (C.c_void_p * max(1, nb))(*[C.c_void_p(p) for p in buffer_ptrs])
    la = (C.c_int64 * max(1, nb))(*row_pitch)
    return int(lib().dag_run_noalloc(na, nn, ba, nb, pa, la, C.byref(options) if options else None,
                                     C.c_void_p(stream)))


def dag_trace_launch(h):
    """(first CTA entry, last CTA exit) of the last traced persistent launch, ns."""
    out = (u64 * 2)()
    check(lib().dag_trace_launch(h, out), "dag_trace_launch")
    return int(out[0]), int(out[1])


def dag_plan_get(h) -> dag_plan_info:
    info = dag_plan_info()
    check(lib().dag_plan_get(h, C.byref(info)), "dag_plan_get")
    return info


def dag_node_costs_get(h):
    import numpy as np
    n = C.c_int(0)
    check(lib().dag_node_costs_get(h, None, 0, C.byref(n)), "dag_node_costs_get")
    out = np.empty(max(1, n.value), np.float32)
    check(lib().dag_node_costs_get(h, out.ctypes.data, n.value, C.byref(n)), "dag_node_costs_get")
    return out[: n.value]


def dag_tiles_get(h):
    import numpy as np
    n = C.c_int(0)
    check(lib().dag_tiles_get(h, None, 0, C.byref(n)), "dag_tiles_get")
    out = (i32 * (6 * max(1, n.value)))()
    check(lib().dag_tiles_get(h, out, n.value, C.byref(n)), "dag_tiles_get")
    return np.frombuffer(out, dtype=np.int32)[: 6 * n.value].reshape(-1, 6).copy()


def dag_set_device(ordinal: int) -> None:
    check(lib().dag_set_device(ordinal), "dag_set_device")


def dag_set_peaks(bf16_tflops: float, f32_tflops: float, hbm_gbs: float) -> None:
    lib().dag_set_peaks(bf16_tflops, f32_tflops, hbm_gbs)


# learned cost model -------------------------------------------------------------
def _f32(a):
    import numpy as np
    return np.ascontiguousarray(a, dtype=np.float32)


def dag_mlp_create(in_dim: int):
    h = C.c_void_p()
    check(lib().dag_mlp_create(in_dim, C.byref(h)), "dag_mlp_create")
    return h


def dag_mlp_param_count(m) -> int:
    return int(lib().dag_mlp_param_count(m))


def dag_mlp_set_params(m, params) -> None:
    p = _f32(params)
    check(lib().dag_mlp_set_params(m, p.ctypes.data, p.size), "dag_mlp_set_params")


def dag_mlp_get_params(m):
    import numpy as np
    p = np.empty(dag_mlp_param_count(m), np.float32)
    check(lib().dag_mlp_get_params(m, p.ctypes.data, p.size), "dag_mlp_get_params")
    return p


def dag_mlp_loss_grad(m, X, y):
    import numpy as np
    X, y = _f32(X), _f32(y)
    g = np.empty(dag_mlp_param_count(m), np.float32)
    loss = C.c_float(0)
    check(lib().dag_mlp_loss_grad(m, X.ctypes.data, y.ctypes.data, len(y), C.byref(loss), g.ctypes.data),
          "dag_mlp_loss_grad")
    return float(loss.value), g


def dag_mlp_train(m, X, y, steps: int, batch: int, lr: float) -> None:
    X, y = _f32(X), _f32(y)
    check(lib().dag_mlp_train(m, X.ctypes.data, y.ctypes.data, len(y), steps, batch, lr), "dag_mlp_train")


def dag_mlp_predict(m, X):
    import numpy as np
    X = _f32(X)
    out = np.empty(X.shape[0], np.float32)
    check(lib().dag_mlp_predict(m, X.ctypes.data, X.shape[0], out.ctypes.data), "dag_mlp_predict")
    return out


def dag_mlp_destroy(m) -> None:
    check(lib().dag_mlp_destroy(m), "dag_mlp_destroy")


# serving -----------------------------------------------------------------------
def dag_poll(h) -> int:
    return int(lib().dag_poll(h))


def _ptrs(ps):
    return (C.c_void_p * max(1, len(ps)))(*[C.c_void_p(p) if p else None for p in ps])


def dag_server_create(models, max_slots: int, hbm_reserve_bytes: int = 0, options: Optional[dag_options] = None):
    """models: list of (nodes, buffers, weights_ptrs, node_cost_us or None)."""
    keep = []
    arr = (dag_model_desc * len(models))()
    for i, (nodes, bufs, wptrs, costs) in enumerate(models):
        na, nn = _arr(dag_node_desc, nodes)
        ba, nb = _arr(dag_buffer_desc, bufs)
        wa = _ptrs(wptrs)
        ca = (f32 * len(costs))(*costs) if costs is not None else None
        keep += [na, ba, wa, ca]
        arr[i] = dag_model_desc(C.cast(na, C.POINTER(dag_node_desc)), nn, C.cast(ba, C.POINTER(dag_buffer_desc)), nb,
                                C.cast(wa, C.POINTER(C.c_void_p)),
                                C.cast(ca, C.POINTER(f32)) if ca is not None else None)
    h = C.c_void_p()
    check(lib().dag_server_create(arr, len(models), max_slots, hbm_reserve_bytes,
                                  C.byref(options) if options else None, C.byref(h)), "dag_server_create")
    return h


def dag_server_set_io(s, model: int, inputs, outputs) -> None:
    check(lib().dag_server_set_io(s, model, _ptrs(inputs), _ptrs(outputs)), "dag_server_set_io")


def dag_server_warm(s, model: int, n_slots: int) -> None:
    check(lib().dag_server_warm(s, model, n_slots), "dag_server_warm")


def dag_server_submit(s, model: int, inputs=None, outputs=None) -> int:
    t = C.c_uint64(0)
    check(lib().dag_server_submit(s, model, _ptrs(inputs) if inputs is not None else None,
                                  _ptrs(outputs) if outputs is not None else None, C.byref(t)), "dag_server_submit")
    return t.value


def dag_server_progress(s) -> int:
    return int(lib().dag_server_progress(s))


def dag_server_wait(s, ticket: int, timeout_ns: int = 60_000_000_000):
    info = dag_request_info()
    check(lib().dag_server_wait(s, ticket, timeout_ns, C.byref(info)), "dag_server_wait")
    return info


def dag_server_simulate(s, model_seq, rate_hz: float, seed: int):
    import numpy as np
    n = len(model_seq)
    ms = (i32 * n)(*model_seq)
    lat = np.zeros(n, np.float64)
    wall = C.c_double(0)
    mif = C.c_int(0)
    check(lib().dag_server_simulate(s, ms, n, rate_hz, seed, lat.ctypes.data_as(C.POINTER(C.c_double)),
                                    C.byref(wall), C.byref(mif)), "dag_server_simulate")
    return lat, wall.value, mif.value


def dag_server_slots(s) -> int:
    return int(lib().dag_server_slots(s))


def dag_server_destroy(s) -> None:
    check(lib().dag_server_destroy(s), "dag_server_destroy")
