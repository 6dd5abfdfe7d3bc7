"""PyTorch-facing API of libtnet: device memory, streams and autograd glue.

Every step of the computation runs in libtnet's CUDA kernels; this module
only allocates tensors, packs the weight blob in the layout of
include/tnet.h and passes pointers and the current stream.
"""
from __future__ import annotations

import ctypes
import dataclasses
import json
import os

import numpy as np
import torch

from . import _lib

# Parameter order of the weight blob (include/tnet.h).
def blob_layout(F: int, K: int, L: int, max_z: int) -> list[tuple[str, tuple[int, ...]]]:
    out = [("emb", (max_z, F)), ("emb2_w", (F, 2 * F)), ("emb2_b", (F,)),
           ("dproj_w", (3, F, K)), ("dproj_b", (3, F)), ("emb_ln_g", (F,)), ("emb_ln_b", (F,)),
           ("emb_mlp1_w", (2 * F, F)), ("emb_mlp1_b", (2 * F,)),
           ("emb_mlp2_w", (3 * F, 2 * F)), ("emb_mlp2_b", (3 * F,)), ("emb_mix_w", (3, F, F))]
    for l in range(L):
        out += [(f"l{l}_mlp1_w", (F, K)), (f"l{l}_mlp1_b", (F,)),
                (f"l{l}_mlp2_w", (2 * F, F)), (f"l{l}_mlp2_b", (2 * F,)),
                (f"l{l}_mlp3_w", (3 * F, 2 * F)), (f"l{l}_mlp3_b", (3 * F,)),
                (f"l{l}_mix1_w", (3, F, F)), (f"l{l}_mix2_w", (3, F, F))]
    out += [("out_ln_g", (3 * F,)), ("out_ln_b", (3 * F,)), ("out_w", (F, 3 * F)), ("out_b", (F,)),
            ("head1_w", (F // 2, F)), ("head1_b", (F // 2,)), ("head2_w", (1, F // 2)), ("head2_b", (1,))]
    return out


def pack_weights(weights: dict, F: int, K: int, L: int, max_z: int) -> np.ndarray:
    parts = []
    for name, shp in blob_layout(F, K, L, max_z):
        a = np.asarray(weights[name], dtype=np.float32)
        if a.shape != shp:
            raise ValueError(f"{name}: shape {a.shape}, expected {shp}")
        parts.append(a.ravel())
    return np.concatenate(parts)


def unpack_weights(blob, F: int, K: int, L: int, max_z: int) -> dict:
    blob = np.asarray(blob)
    out, o = {}, 0
    for name, shp in blob_layout(F, K, L, max_z):
        n = int(np.prod(shp))
        out[name] = blob[o:o + n].reshape(shp)
        o += n
    return out


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


@dataclasses.dataclass
class NeighborList:
    row_ptr: torch.Tensor   # [N+1] int32
    col: torch.Tensor       # [cap] int32
    n_pairs: torch.Tensor   # [1] int64 (device)
    cutoff: float


class TensorNet:
    """One libtnet context: model shape, limits and its device workspace."""

    def __init__(self, weights: dict, F=128, K=32, L=2, max_z=100, cutoff_upper=5.0, cutoff_lower=0.0,
                 max_atoms=1024, max_systems=1, max_pairs=65536, precision=0, device="cuda",
                 recompute_edges=False, radial_table=0):
        self.lib = _lib.load()
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise RuntimeError("libtnet runs on CUDA devices only")
        self.F, self.K, self.L, self.max_z = F, K, L, max_z
        self.cutoff = float(cutoff_upper)
        self.desc = _lib.ModelDesc(F, K, L, max_z, cutoff_upper, cutoff_lower, precision, int(bool(recompute_edges)),
                                   int(radial_table))
        self.max_atoms, self.max_systems, self.max_pairs = int(max_atoms), int(max_systems), int(max_pairs)
        nbytes = self.lib.tnet_workspace_bytes(ctypes.byref(self.desc), self.max_atoms, self.max_systems,
                                               self.max_pairs)
        if nbytes < 0:
            raise ValueError("invalid model shape or limits")
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=self.device)
            base = self.workspace.data_ptr()
            aligned = (base + 255) & ~255
            self.ctx = ctypes.c_void_p()
            _lib.check(self.lib.tnet_create(ctypes.byref(self.ctx), ctypes.byref(self.desc), self.max_atoms,
                                            self.max_systems, self.max_pairs, ctypes.c_void_p(aligned),
                                            int(nbytes)), "tnet_create")
        self.n_weights = int(self.lib.tnet_weights_count(ctypes.byref(self.desc)))
        self.set_weights(weights)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and ctx.value:
            self.lib.tnet_destroy(ctx)
            self.ctx = None

    def set_weights(self, weights) -> None:
        if isinstance(weights, torch.Tensor):
            w = weights.detach().to(self.device, torch.float32).contiguous()
        else:
            w = torch.from_numpy(pack_weights(weights, self.F, self.K, self.L, self.max_z)).to(self.device)
        if w.numel() != self.n_weights:
            raise ValueError("weight blob size mismatch")
        self.weights = w
        if self.desc.radial_table > 0:   # tabulate the radial functions of these weights
            _lib.check(self.lib.tnet_radial_tables(self.ctx, _p(self.weights), _stream(self.device)),
                       "tnet_radial_tables")

    # -------------------------------------------------------------- tuning
    def get_tuning(self) -> list[int]:
        n = self.lib.tnet_tuning_knobs()
        buf = (ctypes.c_int32 * n)()
        _lib.check(self.lib.tnet_get_tuning(self.ctx, buf, n), "tnet_get_tuning")
        return list(buf)

    def set_tuning(self, knobs) -> None:
        buf = (ctypes.c_int32 * len(knobs))(*knobs)
        _lib.check(self.lib.tnet_set_tuning(self.ctx, buf, len(knobs)), "tnet_set_tuning")

    # -------------------------------------------------------------- status
    def reset_status(self):
        self.status.zero_()

    def check_status(self, where="libtnet"):
        code = int(self.status.item())
        if code:
            raise _lib.TnetError(code, where)

    # ----------------------------------------------------------- neighbors
    def neighbors(self, pos, batch=None, box=None, n_systems=1, cutoff=None, cap=None,
                  out: NeighborList | None = None) -> NeighborList:
        N = pos.shape[0]
        cutoff = self.cutoff if cutoff is None else float(cutoff)
        cap = self.max_pairs if cap is None else int(cap)
        if out is None:
            out = NeighborList(torch.empty(N + 1, dtype=torch.int32, device=self.device),
                               torch.empty(max(cap, 1), dtype=torch.int32, device=self.device),
                               torch.zeros(1, dtype=torch.int64, device=self.device), cutoff)
        _lib.check(self.lib.tnet_neighbors(self.ctx, N, n_systems, _p(pos), _p(batch), _p(box),
                                           ctypes.c_float(cutoff), _p(out.row_ptr), _p(out.col), cap,
                                           _p(out.n_pairs), _p(self.status), _stream(self.device)),
                   "tnet_neighbors")
        return out

    # ------------------------------------------------------- energy/forces
    def energy_forces(self, z, pos, nl: NeighborList, batch=None, box=None, n_systems=1, forces=True,
                      grad_weights=False, seed=None, out=None):
        N = pos.shape[0]
        if out is None:
            E = torch.empty(n_systems, dtype=torch.float64, device=self.device)
            Fo = torch.empty((N, 3), dtype=torch.float32, device=self.device) if forces else None
            G = torch.empty(self.n_weights, dtype=torch.float32, device=self.device) if grad_weights else None
        else:
            E, Fo, G = out
        _lib.check(self.lib.tnet_energy_forces(self.ctx, _p(self.weights), N, n_systems, _p(z), _p(pos),
                                               _p(batch), _p(box), _p(nl.row_ptr), _p(nl.col), _p(seed),
                                               _p(E), _p(Fo), _p(G), _p(self.status), _stream(self.device)),
                   "tnet_energy_forces")
        return E, Fo, G

    # ----------------------------------------------------------------- MD
    def md(self, z, inv_mass, pos, vel, box, dt, skin, rebuild_every, n_steps, e_kin=None, e_pot=None):
        N = pos.shape[0]
        e_kin = torch.empty(n_steps, dtype=torch.float64, device=self.device) if e_kin is None else e_kin
        e_pot = torch.empty(n_steps, dtype=torch.float64, device=self.device) if e_pot is None else e_pot
        _lib.check(self.lib.tnet_md_step(self.ctx, _p(self.weights), N, _p(z), _p(inv_mass), _p(pos), _p(vel),
                                         _p(box), ctypes.c_float(dt), ctypes.c_float(skin), int(rebuild_every),
                                         int(n_steps), _p(e_kin), _p(e_pot), _p(self.status),
                                         _stream(self.device)), "tnet_md_step")
        return e_kin, e_pot

    def md_neighbor_list(self, n_atoms: int) -> NeighborList:
        """A copy of the neighbor list md() keeps (cutoff + skin, last rebuild)."""
        nl = NeighborList(torch.empty(n_atoms + 1, dtype=torch.int32, device=self.device),
                          torch.empty(self.max_pairs, dtype=torch.int32, device=self.device),
                          torch.zeros(1, dtype=torch.int64, device=self.device), float("nan"))
        _lib.check(self.lib.tnet_md_neighbor_list(self.ctx, int(n_atoms), _p(nl.row_ptr), _p(nl.col), self.max_pairs,
                                                  _p(nl.n_pairs), _stream(self.device)), "tnet_md_neighbor_list")
        return nl

    def md_rebuilds(self) -> int:
        """Neighbor-list builds of the last md() call (waits for the device)."""
        n = ctypes.c_int64()
        _lib.check(self.lib.tnet_md_rebuilds(self.ctx, ctypes.byref(n)), "tnet_md_rebuilds")
        return int(n.value)


class EnergyFn(torch.autograd.Function):
    """E_s(pos, weights) with gradients from libtnet's reverse pass.

    forward(pos, weights, model, z, nl, batch, box, n_systems) -> E [S] f64.
    d/dpos = -forces scaled per system by the incoming gradient; d/dweights
    comes from a second reverse pass seeded with the incoming gradient."""

    @staticmethod
    def forward(ctx, pos, weights, model: TensorNet, z, nl, batch, box, n_systems):
        model.set_weights(weights)
        E, Fo, _ = model.energy_forces(z, pos.detach(), nl, batch, box, n_systems, forces=True)
        ctx.model, ctx.args = model, (z, nl, batch, box, n_systems)
        ctx.save_for_backward(pos, weights, Fo)
        return E

    @staticmethod
    def backward(ctx, gE):
        pos, weights, Fo = ctx.saved_tensors
        z, nl, batch, box, n_systems = ctx.args
        model = ctx.model
        gpos = gw = None
        if ctx.needs_input_grad[0]:
            scale = gE.to(torch.float32)[batch.long()] if batch is not None else gE.to(torch.float32)[0]
            gpos = -Fo * (scale[:, None] if batch is not None else scale)
        if ctx.needs_input_grad[1]:
            model.set_weights(weights)
            _, _, gw = model.energy_forces(z, pos.detach(), nl, batch, box, n_systems, forces=True,
                                           grad_weights=True, seed=gE.to(torch.float32).contiguous())
        return gpos, gw, None, None, None, None, None, None


# ------------------------------------------------------------------ autotuner
TUNE_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune", "tuning.json")


def tuning_knobs(lib=None) -> list[tuple[str, list[int]]]:
    lib = lib or _lib.load()
    out = []
    for k in range(lib.tnet_tuning_knobs()):
        buf = (ctypes.c_int32 * 8)()
        n = lib.tnet_tuning_candidates(k, buf, 8)
        out.append((lib.tnet_tuning_name(k).decode(), list(buf)[:n]))
    return out


def autotune(model: TensorNet, z, pos, nl: NeighborList, batch=None, box=None, n_systems=1, reps=5,
             cache: str | None = TUNE_CACHE, force=False, passes=3):
    """Pick launch shapes by timing them on this input (coordinate descent
    over the context's knobs, repeated while it changes a knob, CUDA events
    around CUDA-graph replays of whole energy+force calls),
    set them on the model and cache them as JSON keyed by GPU, precision,
    shape and size.  Returns (knobs, {knob: {candidate: ms}})."""
    dev = model.device
    key = "|".join([torch.cuda.get_device_name(dev), f"knobs{len(model.get_tuning())}", f"p{model.desc.precision}",
                    f"F{model.F}L{model.L}",
                    f"N{pos.shape[0]}", f"S{n_systems}", f"E{int(nl.n_pairs.item()) // 1024}k"])
    table = {}
    if cache and os.path.exists(cache):
        try:
            table = json.load(open(cache))
        except (OSError, ValueError):
            table = {}
    if not force and key in table:
        model.set_tuning(table[key]["knobs"])
        return table[key]["knobs"], table[key].get("timings", {})
    E = torch.empty(n_systems, dtype=torch.float64, device=dev)
    Fo = torch.empty((pos.shape[0], 3), dtype=torch.float32, device=dev)

    def run_ms():
        # as a CUDA-graph replay, the way graph-captured steps run (the knobs
        # are baked into a graph's launches at capture time)
        def call():
            model.energy_forces(z, pos, nl, batch, box, n_systems, out=(E, Fo, None))
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            call()
        torch.cuda.current_stream(dev).wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            call()
        g.replay()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(reps):
            g.replay()
        ev[1].record()
        torch.cuda.synchronize()
        del g
        return ev[0].elapsed_time(ev[1]) / reps

    knobs = model.get_tuning()
    timings = {}
    # knobs interact (programmatic launch changes which grid sizes win), so the
    # descent sweeps again while a sweep still changes something (at most
    # `passes` sweeps)
    for _ in range(passes):
        before = list(knobs)
        for k, (name, cands) in enumerate(tuning_knobs(model.lib)):
            res = {}
            for v in cands:
                trial = list(knobs)
                trial[k] = v
                model.set_tuning(trial)
                res[v] = run_ms()
            knobs[k] = min(res, key=res.get)
            timings[name] = {str(v): round(t, 4) for v, t in res.items()}
        if knobs == before:
            break
    model.set_tuning(knobs)
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        table[key] = {"knobs": knobs, "timings": timings}
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    return knobs, timings
