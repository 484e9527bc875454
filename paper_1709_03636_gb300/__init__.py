"""GB300 tensor-network contraction of QAOA Max-Cut circuits (qTorch method).

Thin Python layer over the C ABI of ``libqtc.so`` (``include/qtc.h``): it
marshals arguments and owns the device arena (a torch tensor); every step of
the contraction runs in the library's CUDA kernels.  PyTorch is used only for
device memory, streams and ``autograd``.
"""

from __future__ import annotations

import ctypes

from ._lib import (QtcError, check, lib, qtc_batch_info, qtc_observable, qtc_plan_info,
                   qtc_plan_opts)

__all__ = [
    "QtcError", "Engine", "Circuit", "Network", "Plan", "Batch", "DTYPES", "ORDERINGS",
    "contract", "qaoa_expectation", "qaoa_expectation_device", "QAOAExpectation",
    "statevector_expectation", "statevector_expectation_device", "optimize_angles",
    "answer_string", "autotune", "shard", "allreduce_sum",
    "GATES",
]

DTYPES = {"c128": 0, "c64": 1, "split_bf16": 2}
ORDERINGS = {"stoch": 0, "lg": 1}
GATES = {"h": 0, "x": 1, "y": 2, "z": 3, "rx": 4, "rz": 5, "zz": 6, "cnot": 7,
         "depolarize": 8, "dephase": 9, "ampdamp": 10}
OBS = {"zz": 0, "identity": 1, "pauli": 2, "amplitude": 3, "projector": 4}


def _dtype(d):
    return DTYPES[d] if isinstance(d, str) else int(d)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _i32(values):
    arr = (ctypes.c_int32 * len(values))(*[int(v) for v in values])
    return arr


def _f64(values):
    return (ctypes.c_double * len(values))(*[float(v) for v in values])


class _Handle:
    _destroy = None

    def __init__(self, ptr):
        self._ptr = ptr

    @property
    def ptr(self):
        return self._ptr

    def close(self):
        if self._ptr:
            getattr(lib, self._destroy)(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Engine(_Handle):
    """One CUDA device plus a caller-owned device arena (a torch uint8 tensor)."""

    _destroy = "qtc_engine_destroy"

    def __init__(self, device: int = 0, arena_bytes: int = 256 << 20, arena=None):
        import torch
        if arena is None:
            arena = torch.empty(arena_bytes, dtype=torch.uint8, device=f"cuda:{device}")
        self.arena = arena
        h = ctypes.c_void_p()
        check(lib.qtc_engine_create(device, ctypes.c_void_p(arena.data_ptr()),
                                    arena.numel() * arena.element_size(), ctypes.byref(h)))
        super().__init__(h)
        self.device = device
        self.graph_options = (False, 0)
        self.task_options = (16, 32768, 1, False)

    def reset(self):
        check(lib.qtc_engine_reset(self.ptr))

    def set_limits(self, max_wave_bytes=8 << 30, wait_limit_ms=10000.0):
        """Graph-executor limits: global intermediates per launch, wait bound."""
        check(lib.qtc_engine_set_limits(self.ptr, int(max_wave_bytes), float(wait_limit_ms)))

    def set_graph_options(self, force_graph=False, small_rank=0):
        """Run small networks through the graph executor / move tensors of
        rank > small_rank to global memory (0: default)."""
        check(lib.qtc_engine_set_graph_options(self.ptr, int(force_graph), int(small_rank)))
        self.graph_options = (bool(force_graph), int(small_rank))

    def set_task_options(self, task_terms_log2=16, subtree_bytes=32768, warp_teams=1,
                         graph_hi_occupancy=False):
        """Task shapes: about 2^task_terms_log2 multiply-adds per graph chunk
        task, at most subtree_bytes of values per shared-memory subtree, how
        small networks run (0: one per CTA; 1: one per warp where it fits;
        2: one per warp with the steps streamed from global memory), and the
        graph executor's five-CTAs-per-SM build (complex64)."""
        check(lib.qtc_engine_set_task_options(self.ptr, int(task_terms_log2),
                                              int(subtree_bytes), int(warp_teams),
                                              int(bool(graph_hi_occupancy))))
        self.task_options = (int(task_terms_log2), int(subtree_bytes), int(warp_teams),
                             bool(graph_hi_occupancy))

    def set_tile_mode(self, mode=1):
        """Graph executor: 0 row/split chunk paths only, 1 tiles for steps
        with both operands in global memory and long reductions, 2 tiles for
        every step that tiles (footprints staged through shared memory)."""
        check(lib.qtc_engine_set_tile_mode(self.ptr, int(mode)))

    @property
    def last_launches(self) -> int:
        return lib.qtc_engine_last_launches(self.ptr)


class Circuit(_Handle):
    _destroy = "qtc_circuit_destroy"

    def __init__(self, n: int, n_params: int, _ptr=None):
        if _ptr is None:
            h = ctypes.c_void_p()
            check(lib.qtc_circuit_create(n, n_params, ctypes.byref(h)))
            _ptr = h
        super().__init__(_ptr)
        self.n = n
        self.n_params = n_params
        self.edges = None
        self.p = 0

    @classmethod
    def qaoa(cls, n: int, edges, p: int, noise=None) -> "Circuit":
        """Section 4.1 circuit: H, then p x (ZZ(gamma_k) per edge, RX(2 beta_k)).
        noise = (channel, strength), channel in "depolarize", "dephase",
        "ampdamp": that channel on every qubit after each layer's mixer."""
        flat = [v for e in edges for v in e]
        h = ctypes.c_void_p()
        if noise is None:
            check(lib.qtc_circuit_qaoa(n, _i32(flat), len(edges), p, ctypes.byref(h)))
        else:
            kind, strength = noise
            check(lib.qtc_circuit_qaoa_noisy(n, _i32(flat), len(edges), p, GATES[kind],
                                             float(strength), ctypes.byref(h)))
        c = cls(n, 2 * p, _ptr=h)
        c.edges = [tuple(e) for e in edges]
        c.p = p
        return c

    def add_gate(self, gate, qubits, slot: int = -1, coeff: float = 0.0, constant: float = 0.0):
        g = GATES[gate] if isinstance(gate, str) else int(gate)
        check(lib.qtc_circuit_add_gate(self.ptr, g, _i32(qubits), slot, coeff, constant))
        return self


class Network(_Handle):
    _destroy = "qtc_network_destroy"

    def __init__(self, circuit: Circuit, observable="zz", *, edge=None, pauli=None, bits=None,
                 lightcone: bool = True, diag: bool = True):
        obs = qtc_observable()
        obs.kind = OBS[observable]
        keep = []
        if observable == "zz":
            obs.u, obs.v = edge
        elif observable == "pauli":
            s = pauli.encode()
            keep.append(s)
            obs.pauli = s
        elif observable in ("amplitude", "projector"):
            arr = (ctypes.c_uint8 * len(bits))(*[int(b) for b in bits])
            keep.append(arr)
            obs.bits = ctypes.cast(arr, ctypes.POINTER(ctypes.c_uint8))
        h = ctypes.c_void_p()
        check(lib.qtc_network_build(circuit.ptr, ctypes.byref(obs), int(lightcone), int(diag),
                                    ctypes.byref(h)))
        super().__init__(h)
        self.n_params = circuit.n_params

    def leaves(self):
        """List of dicts (kind, conj, slot, coeff, constant, labels) per leaf."""
        counts = (ctypes.c_int32 * 2)()
        check(lib.qtc_network_leaves(self.ptr, counts, None, None, None, None, None, None))
        n = counts[0]
        kind, conj, slot = ((ctypes.c_int32 * n)() for _ in range(3))
        coeff, const = (ctypes.c_double * n)(), (ctypes.c_double * n)()
        labels = (ctypes.c_int32 * (4 * n))()
        check(lib.qtc_network_leaves(self.ptr, counts, kind, conj, slot, coeff, const, labels))
        return [dict(kind=kind[i], conj=conj[i], slot=slot[i], coeff=coeff[i],
                     constant=const[i], labels=[l for l in labels[4 * i:4 * i + 4] if l >= 0])
                for i in range(n)], counts[1]


    def leaf_values(self, leaf: int, params=()):
        """Leaf `leaf` as the executors build it, at `params` (host): its 2^rank
        elements and their derivatives with respect to its parameter, complex
        numpy arrays indexed like the element index (bit k = label k)."""
        import numpy as np
        val = (ctypes.c_double * (2 * 16))()
        der = (ctypes.c_double * (2 * 16))()
        p = _f64(list(params) + [0.0]) if len(params) else None
        check(lib.qtc_network_leaf_values(self.ptr, int(leaf), p, val, der))
        n = 1 << len(self.leaves()[0][leaf]["labels"])
        v = np.array(val[:2 * n]).view(np.complex128)
        d = np.array(der[:2 * n]).view(np.complex128)
        return v, d


def plan_opts(ordering="lg", seed=0, max_rejections=10, restarts=8, budget_ms=0.0):
    o = qtc_plan_opts()
    o.kind = ORDERINGS[ordering] if isinstance(ordering, str) else int(ordering)
    o.seed = seed
    o.max_rejections = max_rejections
    o.restarts = restarts
    o.budget_ms = budget_ms
    return o


class Plan(_Handle):
    _destroy = "qtc_plan_destroy"

    def __init__(self, network: Network, ordering="lg", seed=0, *, like=None, **kw):
        """Ordering search for `network`; with like=<Plan> the contraction tree
        of that plan is reused (same network structure, other values)."""
        h = ctypes.c_void_p()
        if like is not None:
            check(lib.qtc_plan_reuse(like.ptr, network.ptr, ctypes.byref(h)))
        else:
            opts = plan_opts(ordering, seed, **kw)
            check(lib.qtc_plan_create(network.ptr, ctypes.byref(opts), ctypes.byref(h)))
        super().__init__(h)
        self.n_params = network.n_params

    def stats(self) -> dict:
        info = qtc_plan_info()
        check(lib.qtc_plan_stats(self.ptr, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in info._fields_}

    def steps(self):
        n = self.stats()["n_steps"]
        a = (ctypes.c_int32 * n)()
        b = (ctypes.c_int32 * n)()
        check(lib.qtc_plan_steps(self.ptr, a, b))
        return list(zip(a, b))

    def step_shapes(self):
        """(b, x, y, z) of every step: batch, free-in-A, summed, free-in-B
        label counts (Eq. 1 with batch indices kept)."""
        n = self.stats()["n_steps"]
        s = (ctypes.c_int32 * (4 * n))()
        check(lib.qtc_plan_step_shapes(self.ptr, s))
        return [tuple(s[4 * i:4 * i + 4]) for i in range(n)]


class Batch(_Handle):
    """All per-edge <Z_u Z_v> networks of a QAOA circuit, each with its plan."""

    _destroy = "qtc_batch_destroy"

    def __init__(self, circuit: Circuit, obs_edges=None, *, lightcone=True, diag=True,
                 ordering="lg", seed=0, **kw):
        h = ctypes.c_void_p()
        opts = plan_opts(ordering, seed, **kw)
        if obs_edges is None:
            ptr, m = None, 0
            self.edges = list(circuit.edges)
        else:
            flat = [v for e in obs_edges for v in e]
            ptr, m = _i32(flat), len(obs_edges)
            self.edges = [tuple(e) for e in obs_edges]
        check(lib.qtc_batch_create(circuit.ptr, ptr, m, int(lightcone), int(diag),
                                   ctypes.byref(opts), ctypes.byref(h)))
        super().__init__(h)
        self.p = circuit.p
        self.n_params = circuit.n_params

    def stats(self) -> dict:
        info = qtc_batch_info()
        check(lib.qtc_batch_stats(self.ptr, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in info._fields_}

    def program_info(self, dtype="c64", want_grad=False, force_graph=False, small_rank=0,
                     max_wave_bytes=0, smem_limit=0) -> dict:
        """Build and validate the device program on the host (no GPU)."""
        from ._lib import qtc_program_info
        info = qtc_program_info()
        check(lib.qtc_batch_program_info(self.ptr, _dtype(dtype), int(want_grad),
                                         int(force_graph), int(small_rank), int(max_wave_bytes),
                                         int(smem_limit), ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in info._fields_}

    def launch_info(self, engine: Engine, dtype="c64", want_grad=False) -> dict:
        """Grid, block, shared memory, CTAs per SM, launches, TMEM columns."""
        out = (ctypes.c_int32 * 6)()
        check(lib.qtc_batch_launch_info(engine.ptr, self.ptr, _dtype(dtype), int(want_grad), out))
        return dict(zip(["grid", "block", "smem", "per_sm", "launches", "tmem_cols"], out))

    def partition(self, n_parts: int, want_grad: bool = True):
        """Part (0..n_parts-1) of every network, by longest processing time
        first on algorithmic bytes (qtc_batch_partition), and each part's
        bytes."""
        n = len(self.edges)
        parts = (ctypes.c_int32 * n)()
        cost = (ctypes.c_double * n_parts)()
        check(lib.qtc_batch_partition(self.ptr, int(n_parts), int(want_grad), parts, cost))
        return list(parts), list(cost)

    def subset(self, nets) -> "Batch":
        """The networks `nets` of this batch as a batch of their own, with the
        same plans (qtc_batch_subset)."""
        nets = [int(i) for i in nets]
        h = ctypes.c_void_p()
        check(lib.qtc_batch_subset(self.ptr, _i32(nets), len(nets), ctypes.byref(h)))
        sub = Batch.__new__(Batch)
        _Handle.__init__(sub, h)
        sub.edges = [self.edges[i] for i in nets]
        sub.p = self.p
        sub.n_params = self.n_params
        return sub

    def prepare(self, engine: Engine, dtype="c64", want_grad=False, stream=None):
        check(lib.qtc_batch_prepare(engine.ptr, self.ptr, _dtype(dtype), int(want_grad),
                                    _stream(stream)))


def contract(engine: Engine, plan: Plan, params=(), dtype="c64", want_grad=False, stream=None):
    """Scalar of one network (and d/dparams when want_grad)."""
    out = (ctypes.c_double * 2)()
    grad = (ctypes.c_double * (2 * plan.n_params))() if want_grad else None
    check(lib.qtc_contract(engine.ptr, plan.ptr, _f64(params) if len(params) else None,
                           _dtype(dtype), _stream(stream), out, grad))
    value = complex(out[0], out[1])
    if not want_grad:
        return value
    return value, [complex(grad[2 * k], grad[2 * k + 1]) for k in range(plan.n_params)]


def qaoa_expectation(engine: Engine, batch: Batch, gammas, betas, dtype="c64",
                     want_grad=False, stream=None):
    """(<C>, per-edge <Z_u Z_v>, d<C>/d(gamma, beta) or None), host in and out."""
    p = len(gammas)
    C = ctypes.c_double()
    per_edge = (ctypes.c_double * len(batch.edges))()
    grad = (ctypes.c_double * (2 * p))() if want_grad else None
    check(lib.qtc_qaoa_expectation(engine.ptr, batch.ptr, _f64(gammas), _f64(betas),
                                   _dtype(dtype), int(want_grad), _stream(stream),
                                   ctypes.byref(C), per_edge, grad))
    return C.value, list(per_edge), (list(grad) if want_grad else None)


def qaoa_expectation_device(engine: Engine, batch: Batch, params_dev, out_dev, dtype="c64",
                            want_grad=False, stream=None):
    """Asynchronous form: params_dev (2p float64 CUDA tensor) -> out_dev
    (2 + 2p + m float64 CUDA tensor: <C>, gradient, per-edge <Z_u Z_v>,
    status (0, or 3 when a bounded device wait expired))."""
    check(lib.qtc_qaoa_expectation_device(
        engine.ptr, batch.ptr, ctypes.c_void_p(params_dev.data_ptr()), _dtype(dtype),
        int(want_grad), _stream(stream), ctypes.c_void_p(out_dev.data_ptr())))
    return out_dev


def statevector_expectation(engine: Engine, circuit: Circuit, gammas, betas, dtype="c64",
                            per_edge=False, stream=None):
    """<C> (and per-edge <Z_a Z_b>) from the full 2^n state vector on the GPU."""
    C = ctypes.c_double()
    pe = (ctypes.c_double * len(circuit.edges))() if per_edge else None
    check(lib.qtc_statevector_qaoa(engine.ptr, circuit.ptr, _f64(gammas), _f64(betas),
                                   _dtype(dtype), int(per_edge), _stream(stream),
                                   ctypes.byref(C), pe))
    return C.value, (list(pe) if per_edge else None)


def statevector_expectation_device(engine: Engine, circuit: Circuit, params_dev, out_dev,
                                   dtype="c64", per_edge=False, stream=None):
    """Asynchronous form: out_dev (1 + m float64) = [<C>, <Z_a Z_b> per edge]."""
    check(lib.qtc_statevector_qaoa_device(engine.ptr, circuit.ptr,
                                          ctypes.c_void_p(params_dev.data_ptr()), _dtype(dtype),
                                          int(per_edge), _stream(stream),
                                          ctypes.c_void_p(out_dev.data_ptr())))
    return out_dev


def _autograd():
    import torch

    class QAOAExpectation(torch.autograd.Function):
        """<C>(gamma, beta) with the adjoint-sweep gradient in backward."""

        @staticmethod
        def forward(ctx, params, engine, batch, dtype="c64"):
            p = batch.p
            prm = params.detach().to(device=f"cuda:{engine.device}", dtype=torch.float64)
            prm = prm.contiguous()
            out = torch.empty(2 + 2 * p + len(batch.edges), dtype=torch.float64,
                              device=prm.device)
            qaoa_expectation_device(engine, batch, prm, out, dtype, want_grad=True)
            ctx.save_for_backward(out[1:1 + 2 * p].clone())
            ctx.param_device = params.device
            return out[0].clone().to(device=params.device, dtype=params.dtype)

        @staticmethod
        def backward(ctx, grad_out):
            (grad,) = ctx.saved_tensors
            g = grad.to(device=ctx.param_device, dtype=grad_out.dtype)
            return grad_out * g, None, None, None

    return QAOAExpectation


def answer_string(engine: Engine, circuit: Circuit, params, dtype="c128", ordering="lg",
                  seed=0, stream=None):
    """Section 3.3's estimate of a likely output bit string (the library's
    qtc_answer_string): qubit by qubit, the prefix probability with the
    current qubit projected on |0> against the rest, keeping the likelier
    value (an exact tie is broken by a generator seeded with `seed`).  All n
    contractions share one contraction tree.  Returns (bits, probabilities of
    each chosen prefix).  The circuit may hold noise channels."""
    n = circuit.n
    bits = (ctypes.c_uint8 * n)()
    probs = (ctypes.c_double * n)()
    opts = plan_opts(ordering, seed)
    check(lib.qtc_answer_string(engine.ptr, circuit.ptr, _f64(params) if len(params) else None,
                                _dtype(dtype), ctypes.byref(opts), int(seed), _stream(stream),
                                bits, probs))
    return list(bits), list(probs)


def optimize_angles(engine: Engine, batch: Batch, gammas, betas, *, steps: int = 200,
                    lr: float = 0.05, dtype="c64", tol: float = 1e-9):
    """Maximise <C>(gamma, beta) with Adam on the adjoint gradient (the loop
    the paper drives with NLopt, Section 4.1): every step is one launch of
    the executor for <C> and d<C>/d(gamma, beta).  Returns (best <C>, gammas,
    betas, history of <C>).  Stops early when <C> changes by less than tol
    (relative) over 10 steps."""
    import torch
    p = len(gammas)
    x = torch.tensor(list(gammas) + list(betas), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([x], lr=lr)
    hist = []
    best = (-float("inf"), None)
    for _ in range(steps):
        opt.zero_grad()
        c = QAOAExpectation.apply(x, engine, batch, dtype)
        (-c).backward()
        hist.append(float(c.detach()))
        if hist[-1] > best[0]:
            best = (hist[-1], x.detach().clone())
        opt.step()
        if len(hist) > 10 and abs(hist[-1] - hist[-11]) <= tol * abs(hist[-1]):
            break
    xb = best[1].tolist()
    return best[0], xb[:p], xb[p:], hist


class _LazyAutograd:
    _cls = None

    def apply(self, *args):
        if _LazyAutograd._cls is None:
            _LazyAutograd._cls = _autograd()
        return _LazyAutograd._cls.apply(*args)


QAOAExpectation = _LazyAutograd()


from .shard import allreduce_sum, shard  # noqa: E402  (edge sharding over ranks)
from .tuning import autotune  # noqa: E402  (graph-executor task shapes)
