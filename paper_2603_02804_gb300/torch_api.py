"""PyTorch integration: a simulator object, a ``torch.autograd.Function`` and an
``nn.Module`` for the hardware-efficient ansatz.

PyTorch supplies device memory (the workspace is one uint8 tensor from the
caching allocator) and the current CUDA stream; every step of the simulation
runs in the library's kernels. Autograd integration follows Sec. 3.3's
out-of-place discipline: the forward keeps its checkpoints in the simulator's
workspace and the backward consumes them; if another forward ran on the same
simulator in between, the backward recomputes its forward first.
"""
from __future__ import annotations

import itertools

import torch

from . import qfuse

_PATHS = {"fused": qfuse.QF_PATH_FUSED, "per_gate": qfuse.QF_PATH_PER_GATE}
_ENT = {"chain": qfuse.QF_ENT_CHAIN, "ring": qfuse.QF_ENT_RING}
_LOSS = {"sum": qfuse.QF_LOSS_SUM, "mse": qfuse.QF_LOSS_MSE}
_ENC = {"angles": qfuse.QF_ENC_RY_X, "state": qfuse.QF_ENC_STATE_IN}
_PREC = {"complex64": qfuse.QF_PREC_C64, "complex128": qfuse.QF_PREC_C128}
_ids = itertools.count(1)


def _cuda_check():
    if not torch.cuda.is_available():
        raise RuntimeError("qfuse needs a CUDA device (GB300, sm_103a); there is no CPU fallback")


class Simulator:
    """A planned circuit with its workspace.

    ``n``/``d`` build the hardware-efficient ansatz; ``gates`` (rows of
    (kind, q0, q1, param)) with ``n_params`` builds a user circuit instead.
    ``ckpt_mode`` 0 reverses psi in the adjoint passes between checkpoints;
    1 re-runs each checkpoint block's forward storing the pass outputs
    (bfloat16 with ``mem_save``), as in the paper's checkpointed scheme.
    ``tc_path`` runs the forward rounds as split-precision blocks on the
    tensor cores (12-qubit tiles, n >= 12). ``precision="complex128"``
    simulates complex128 states in float64 arithmetic; theta, x (and y) are
    then float64 (states: complex128) and the *64 entry points run.
    ``program=1`` forces generic steps where round programs would be used.
    ``catch_up`` (0 planner's choice, 1 strict, 2 rising) and ``fwd_ctas``
    (0 automatic, 2, 3) are tuning knobs that leave the results unchanged
    (``autotune.Autotuner`` picks them).
    """

    def __init__(self, n: int, d: int = 0, batch: int = 1, *, entangler: str = "chain", path: str = "fused",
                 tile_bits: int = 0, ckpt_layers: int = 0, gates=None, n_params: int = 0, obs="Z",
                 device=None, ckpt_mode: int = 0, mem_save: bool = False, tc_path: bool = False,
                 encoding: str = "angles", host_staging: bool = True, precision: str = "complex64",
                 program: int = 0, catch_up: int = 0, fwd_ctas: int = 0):
        _cuda_check()
        self.device = torch.device(device or "cuda")
        self.encoding = encoding
        self.f64 = _PREC[precision] == qfuse.QF_PREC_C128
        self.real = torch.float64 if self.f64 else torch.float32
        self.cplx = torch.complex128 if self.f64 else torch.complex64
        if gates is None:
            self.handle = qfuse.qf_hea_create(n, d, _ENT[entangler], _ENC[encoding])
            self.n_params = 3 * n * d
        else:
            self.handle = qfuse.qf_circuit_create(n, gates, n_params, _ENC[encoding])
            self.n_params = n_params
        self.n, self.d = n, d
        self.path = path
        self.obs = qfuse.pauli(obs, n) if not isinstance(obs, qfuse.qf_pauli) else obs
        with torch.cuda.device(self.device):
            self.ws_bytes = qfuse.qf_plan(self.handle, batch, _PATHS[path], tile_bits, ckpt_layers,
                                          ckpt_mode=ckpt_mode, mem_save=mem_save, tc_path=tc_path,
                                          host_staging=host_staging, precision=_PREC[precision], program=program,
                                          catch_up=catch_up, fwd_ctas=fwd_ctas)
            self.ws = torch.empty(max(self.ws_bytes, 1), dtype=torch.uint8, device=self.device)
        self.batch = batch
        self._fwd_id = 0

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                qfuse.qf_circuit_destroy(h)
            except Exception:
                pass
            self.handle = None

    def info(self) -> dict:
        return qfuse.qf_plan_info(self.handle)

    def launches(self) -> int:
        return qfuse.qf_launch_count(self.handle)

    def graph_stats(self) -> dict:
        """Train steps this simulator recorded as CUDA graphs and replayed from one
        ({"recorded": r, "replayed": n}); a loop on fixed buffers replays every
        step from the second on."""
        return qfuse.qf_graph_stats(self.handle)

    def _stream(self):
        return torch.cuda.current_stream(self.device)

    def _check(self, theta, x):
        if self.encoding == "state":
            # initial states [B, 2^n] (passed to the library as (re, im) pairs)
            if x.dtype != self.cplx or x.dim() != 2 or x.shape[1] != 1 << self.n:
                raise TypeError(f"x must be {self.cplx} [B, 2^n] initial states")
        elif x.dtype != self.real or x.dim() != 2 or x.shape[1] != self.n:
            raise TypeError(f"x must be {self.real} [B, n] encoding angles")
        if theta.dtype != self.real:
            raise TypeError(f"theta must be {self.real}")
        if not (theta.is_cuda and x.is_cuda and theta.is_contiguous() and x.is_contiguous()):
            raise ValueError("theta and x must be contiguous CUDA tensors")
        if theta.numel() != self.n_params or x.shape[0] > self.batch:
            raise ValueError("shape mismatch with the planned circuit")

    def forward(self, theta: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
        """E_b for every sample (float64 [B])."""
        self._check(theta, x)
        B = x.shape[0]
        E = torch.empty(B, dtype=torch.float64, device=self.device)
        fn = qfuse.qf_forward64 if self.f64 else qfuse.qf_forward
        fn(self.handle, theta, x, B, self.obs, E, self.ws, self.ws_bytes, self._stream())
        self._fwd_id = next(_ids)
        return E

    def backward(self, theta, x, dLdE, per_sample: bool = False) -> torch.Tensor:
        """Adjoint gradient after forward(theta, x): float64 [P] or [B, P]."""
        self._check(theta, x)
        B = x.shape[0]
        dLdE = dLdE.to(device=self.device, dtype=torch.float64).contiguous()
        shape = (B, self.n_params) if per_sample else (self.n_params,)
        g = torch.empty(shape, dtype=torch.float64, device=self.device)
        fn = qfuse.qf_backward64 if self.f64 else qfuse.qf_backward
        fn(self.handle, theta, x, B, self.obs, dLdE, g, per_sample, self.ws, self.ws_bytes, self._stream())
        return g

    def train_step(self, theta, x, y=None, loss: str = "sum", out=None):
        """Forward, loss and backward in one call: (loss [1], E [B], grad [P]) on the device.
        ``out``: float64 device tensors (loss [1], E [>= B], grad [P]) to write (e.g. from
        ``device_outputs()``). The library replays a step from a CUDA graph it recorded
        when the same buffers come back, so reusing inputs and outputs saves launches."""
        self._check(theta, x)
        B = x.shape[0]
        out_loss, E, g = out if out is not None else self.device_outputs(B)
        if (E.numel() < B or g.numel() != self.n_params or E.dtype != torch.float64 or not E.is_cuda
                or not g.is_cuda or not out_loss.is_cuda):
            raise ValueError("out buffers must be float64 CUDA tensors (loss [1], E [>= B], grad [P])")
        if y is not None and (y.dtype != self.real or not y.is_cuda):
            raise TypeError(f"y must be a {self.real} CUDA tensor")
        fn = qfuse.qf_train_step64 if self.f64 else qfuse.qf_train_step
        fn(self.handle, theta, x, y, B, _LOSS[loss], self.obs, out_loss, E, g, self.ws, self.ws_bytes, self._stream())
        self._fwd_id = next(_ids)
        return out_loss, E, g

    def device_outputs(self, batch: int | None = None):
        """Device buffers (loss [1], E [B], grad [P]) for ``train_step(out=...)``."""
        B = self.batch if batch is None else batch
        z = lambda k: torch.empty(k, dtype=torch.float64, device=self.device)
        return z(1), z(B), z(self.n_params)

    def host_outputs(self, batch: int | None = None):
        """Pinned host buffers (loss [1], E [B], grad [P]) for ``train_step_host(out=...)``."""
        B = self.batch if batch is None else batch
        z = lambda k: torch.empty(k, dtype=torch.float64).pin_memory()
        return z(1), z(B), z(self.n_params)

    def train_step_host(self, theta_h, x_h, y_h=None, loss: str = "sum", out=None):
        """The same step from host (ideally pinned) tensors; returns host results.
        ``out``: (loss [1], E [B], grad [P]) float64 host tensors to write
        (e.g. from ``host_outputs()``); pinning them once instead of per call
        saves a host allocation per step."""
        B = x_h.shape[0]
        out_loss, E, g = out if out is not None else self.host_outputs(B)
        if E.numel() < B or g.numel() != self.n_params or E.dtype != torch.float64:
            raise ValueError("out buffers must be float64 (loss [1], E [>= B], grad [P])")
        fn = qfuse.qf_train_step_host64 if self.f64 else qfuse.qf_train_step_host
        fn(self.handle, theta_h, x_h, y_h, B, _LOSS[loss], self.obs, out_loss, E, g, self.ws, self.ws_bytes,
           self._stream())
        self._fwd_id = next(_ids)
        return out_loss, E, g


class QFuseFn(torch.autograd.Function):
    """E = QFuseFn.apply(theta, x, sim): fused forward; backward runs the fused
    adjoint kernels with dL/dE from autograd (Eq. 4's chain-rule seed)."""

    @staticmethod
    def forward(ctx, theta, x, sim: Simulator):
        theta_c = theta.detach().contiguous()
        x_c = x.detach().contiguous()
        E = sim.forward(theta_c, x_c)
        ctx.sim = sim
        ctx.fwd_id = sim._fwd_id
        ctx.save_for_backward(theta_c, x_c)
        return E

    @staticmethod
    def backward(ctx, gE):
        theta, x = ctx.saved_tensors
        sim: Simulator = ctx.sim
        if sim._fwd_id != ctx.fwd_id:  # workspace was reused: recompute this forward
            sim.forward(theta, x)
        g = sim.backward(theta, x, gE)
        return g.to(theta.dtype), None, None


class HEA(torch.nn.Module):
    """Hardware-efficient ansatz with RY(x) encoding, returning <O> per sample."""

    def __init__(self, n: int, d: int, max_batch: int, *, obs="Z", entangler="chain", path="fused",
                 ckpt_layers: int = 0, tile_bits: int = 0, device=None, init=None, precision: str = "complex64"):
        super().__init__()
        self.sim = Simulator(n, d, max_batch, entangler=entangler, path=path, tile_bits=tile_bits,
                             ckpt_layers=ckpt_layers, obs=obs, device=device, precision=precision)
        theta = init if init is not None else torch.rand(3 * n * d, dtype=self.sim.real) * (2 * torch.pi)
        self.theta = torch.nn.Parameter(theta.to(device=self.sim.device, dtype=self.sim.real))

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        return QFuseFn.apply(self.theta, x.to(device=self.sim.device, dtype=self.sim.real), self.sim)


class Batch:
    """Many hardware-efficient-ansatz circuits trained in one persistent launch.

    specs: list of (n_qubits, n_layers, batch). tile_bits: None (12, the
    whole state for n <= 12), an int, or a callable (n, d, B) returning K or
    a dict of plan options (tile_bits, catch_up), e.g. an autotuner's choice.
    Inputs and outputs are concatenated over circuits in spec order (offsets
    from `layout()`).
    """

    def __init__(self, specs, loss: str = "sum", obs="Z", ckpt_layers: int = 0, tile_bits=None, device=None):
        _cuda_check()
        self.device = torch.device(device or "cuda")
        self.specs = [(int(n), int(d), int(B)) for n, d, B in specs]
        self.loss = loss
        self.handles = []
        self.plan_opts = []
        pauli_list = []
        for n, d, B in self.specs:
            h = qfuse.qf_hea_create(n, d, qfuse.QF_ENT_CHAIN)
            self.handles.append(h)
            cfg = tile_bits(n, d, B) if callable(tile_bits) else (tile_bits or 0)
            cfg = cfg if isinstance(cfg, dict) else {"tile_bits": int(cfg)}
            self.plan_opts.append({"tile_bits": int(cfg.get("tile_bits", 0)), "catch_up": int(cfg.get("catch_up", 0))})
            qfuse.qf_plan(h, B, qfuse.QF_PATH_FUSED, self.plan_opts[-1]["tile_bits"], ckpt_layers, host_only=True,
                          catch_up=self.plan_opts[-1]["catch_up"])
            pauli_list.append(qfuse.pauli(obs, n) if not isinstance(obs, qfuse.qf_pauli) else obs)
        with torch.cuda.device(self.device):
            self.handle, self.ws_bytes = qfuse.qf_batch_create(self.handles, [B for _, _, B in self.specs],
                                                               pauli_list, _LOSS[loss])
            self.ws = torch.empty(max(self.ws_bytes, 1), dtype=torch.uint8, device=self.device)
        self.theta_off, self.x_off, self.sample_off = qfuse.qf_batch_layout(self.handle, len(self.specs))
        info = qfuse.qf_batch_info(self.handle)
        self.n_items = info["n_items"]
        self.n_samples = info["n_samples"]
        self.n_params = info["n_params"]
        self._graph_stream = None

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                qfuse.qf_batch_destroy(h)
            except Exception:
                pass
        for c in getattr(self, "handles", []):
            try:
                qfuse.qf_circuit_destroy(c)
            except Exception:
                pass

    def outputs(self):
        z = lambda k: torch.empty(k, dtype=torch.float64, device=self.device)
        return z(1), z(self.n_samples), z(self.n_params)

    def train_step(self, theta, x, y=None, out=None):
        loss, E, g = out if out is not None else self.outputs()
        qfuse.qf_batch_train_step(self.handle, theta, x, y, loss, E, g, self.ws, self.ws_bytes,
                                  torch.cuda.current_stream(self.device))
        return loss, E, g

    def capture(self, theta, x, y, out, stream):
        """Capture one step with these buffers into a CUDA graph (replay())."""
        loss, E, g = out
        self._graph_stream = stream
        qfuse.qf_batch_graph_capture(self.handle, theta, x, y, loss, E, g, self.ws, self.ws_bytes, stream)

    def replay(self):
        qfuse.qf_batch_graph_launch(self.handle, self._graph_stream)
