"""Torch-facing wrapper of the C ABI (device memory and streams come from
PyTorch; every computation runs in the library's CUDA kernels)."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import capi

_EXPORT_DTYPES = {
    capi.EXPORT_Y: torch.float64, capi.EXPORT_DX: torch.float64, capi.EXPORT_DD: torch.float32,
    capi.EXPORT_CT: torch.float32, capi.EXPORT_W: torch.float32, capi.EXPORT_PERM: torch.int32,
    capi.EXPORT_SLOTS: torch.int32, capi.EXPORT_GPTR: torch.int32, capi.EXPORT_WIN: torch.int32,
    capi.EXPORT_COST: torch.float64, capi.EXPORT_PMPOS: torch.int32, capi.EXPORT_PPTR: torch.int32,
}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class DPVBA:
    """A bundle-adjustment handle bound to the current CUDA device and stream.

    ``set_graph`` borrows ``poses`` (float64 [N,7]) and ``patches`` (float32
    [P,3,3,3]), which ``step`` updates in place, and ``targets``/``weights``
    (float32 [E,2]), which are read on every ``step``.  The wrapper keeps
    references to them so they outlive the handle's use.
    """

    def __init__(self, precision: str = "fp32", lambda_pose=1e-4, lambda_depth=1e-4, z_min=0.1, d_min=1e-3,
                 patches_per_group: int = 0, max_refine: int = 3, stream: torch.cuda.Stream | None = None,
                 capture: bool = False, residual_pixels: int = 1, timeout_cycles: int | None = None,
                 dense: str = "auto"):
        self._lib = capi.lib()
        self._h = ctypes.c_void_p()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        extra = {} if timeout_cycles is None else {"timeout_cycles": int(timeout_cycles)}
        extra["dense_policy"] = {"auto": capi.BA_DENSE_AUTO, "always": capi.BA_DENSE_ALWAYS,
                                 "never": capi.BA_DENSE_NEVER}[dense]
        opt = capi.default_options(
            precision=capi.BA_MIXED if precision == "mixed" else capi.BA_FP32, lambda_pose=lambda_pose,
            lambda_depth=lambda_depth, z_min=z_min, d_min=d_min, patches_per_group=patches_per_group,
            max_refine=max_refine, stream=self.stream.cuda_stream, residual_pixels=residual_pixels, **extra)
        self.residual_pixels = residual_pixels
        capi.check(None, self._lib.ba_create(ctypes.byref(self._h), ctypes.byref(opt)))
        self._keep = ()
        self.N = self.P = self.E = 0
        if capture:
            self.set_capture(True)

    # ------------------------------------------------------------------ core
    def set_graph(self, poses, patches, ii, jj, kk, targets, weights, intrinsics):
        for name, t, dt in (("poses", poses, torch.float64), ("patches", patches, torch.float32),
                            ("ii", ii, torch.int32), ("jj", jj, torch.int32), ("kk", kk, torch.int32),
                            ("targets", targets, torch.float32), ("weights", weights, torch.float32),
                            ("intrinsics", intrinsics, torch.float32)):
            if t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
                raise TypeError(f"{name}: need a contiguous CUDA {dt} tensor")
        N, P, E = poses.shape[0], patches.shape[0], ii.shape[0]
        if targets.numel() != 2 * self.residual_pixels * E:
            raise ValueError("targets: [E,2], or [E,9,2] with residual_pixels=9")
        self._keep = (poses, patches, ii, jj, kk, targets, weights, intrinsics)
        self.N, self.P, self.E = N, P, E
        capi.check(self._h, self._lib.ba_set_graph(
            self._h, N, P, E, _ptr(poses), _ptr(patches), _ptr(ii), _ptr(jj), _ptr(kk), _ptr(targets),
            _ptr(weights), _ptr(intrinsics)))

    def set_graph_batched(self, poses, patches, ii, jj, kk, targets, weights, intrinsics, frame_off, patch_off,
                          edge_off):
        """Bind independent problems together: the tensors are the problems'
        arrays concatenated (ii, jj, kk local to each problem), intrinsics is
        float32 [B,4], and the offsets are int sequences of length B+1."""
        for name, t, dt in (("poses", poses, torch.float64), ("patches", patches, torch.float32),
                            ("ii", ii, torch.int32), ("jj", jj, torch.int32), ("kk", kk, torch.int32),
                            ("targets", targets, torch.float32), ("weights", weights, torch.float32),
                            ("intrinsics", intrinsics, torch.float32)):
            if t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
                raise TypeError(f"{name}: need a contiguous CUDA {dt} tensor")
        if targets.numel() != 2 * self.residual_pixels * ii.shape[0]:
            raise ValueError("targets: [E,2], or [E,9,2] with residual_pixels=9")
        offs = [np.ascontiguousarray(np.asarray(o, dtype=np.int64)) for o in (frame_off, patch_off, edge_off)]
        B = len(offs[0]) - 1
        self._keep = (poses, patches, ii, jj, kk, targets, weights, intrinsics, offs)
        self.N, self.P, self.E = poses.shape[0], patches.shape[0], ii.shape[0]
        self.B = B
        lp = ctypes.POINTER(ctypes.c_longlong)
        capi.check(self._h, self._lib.ba_set_graph_batched(
            self._h, B, offs[0].ctypes.data_as(lp), offs[1].ctypes.data_as(lp), offs[2].ctypes.data_as(lp),
            _ptr(poses), _ptr(patches), _ptr(ii), _ptr(jj), _ptr(kk), _ptr(targets), _ptr(weights),
            _ptr(intrinsics)))

    def step(self, iters: int, fixed: int):
        capi.check(self._h, self._lib.ba_step(self._h, iters, fixed))

    def sync(self):
        capi.check(self._h, self._lib.ba_sync(self._h))

    def set_capture(self, on: bool = True):
        """Replay ``step`` from a captured CUDA graph (see ba_set_capture)."""
        capi.check(self._h, self._lib.ba_set_capture(self._h, 1 if on else 0))

    def autotune(self, iters: int, fixed: int, reps: int = 3) -> dict:
        """Time every candidate patch-group size on the bound graph and keep
        the fastest (see ba_autotune); returns the chosen size and the
        candidates' median step times in ms (-1: infeasible)."""
        cap = 16
        groups = (ctypes.c_int * cap)()
        ms = (ctypes.c_float * cap)()
        n = ctypes.c_int()
        best = ctypes.c_int()
        capi.check(self._h, self._lib.ba_autotune(self._h, iters, fixed, reps, cap, groups, ms, ctypes.byref(n),
                                                  ctypes.byref(best)))
        return {"G": best.value, "candidates": {groups[i]: float(ms[i]) for i in range(min(n.value, cap))}}

    def close(self):
        if self._h:
            self._lib.ba_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------------- adjoint
    def set_record(self, on: bool = True):
        """Record the following ``step`` calls as the tape of ``backward``."""
        capi.check(self._h, self._lib.ba_set_record(self._h, 1 if on else 0))

    def backward(self, grad_poses=None, grad_depths=None, initial: bool = False):
        """Reverse-mode pass over the recorded step: returns (grad_targets,
        grad_weights) as float32 [E,2] (grad_targets [E,3,3,2] with
        residual_pixels=9); with ``initial`` also the cotangents of
        the initial state, (grad_tangent0 float64 [N,6], grad_depths0 float32 [P]).
        ``grad_poses`` is float64 [N,7] (d loss / d(t, q) of the final poses),
        ``grad_depths`` float32 [P] (d loss / d final inverse depth)."""
        dev = self._keep[0].device
        if grad_poses is not None:
            grad_poses = grad_poses.to(device=dev, dtype=torch.float64).contiguous()
        if grad_depths is not None:
            grad_depths = grad_depths.to(device=dev, dtype=torch.float32).contiguous()
        gT = torch.empty((self.E, 2) if self.residual_pixels == 1 else (self.E, 3, 3, 2), dtype=torch.float32,
                         device=dev)
        gW = torch.empty((self.E, 2), dtype=torch.float32, device=dev)
        x0 = torch.empty((self.N, 6), dtype=torch.float64, device=dev) if initial else None
        d0 = torch.empty(self.P, dtype=torch.float32, device=dev) if initial else None
        capi.check(self._h, self._lib.ba_backward(self._h, _ptr(grad_poses), _ptr(grad_depths), _ptr(gT), _ptr(gW),
                                                  _ptr(x0), _ptr(d0)))
        return (gT, gW, x0, d0) if initial else (gT, gW)

    # ------------------------------------------------------- loop closure
    def proximity_edges(self, poses, patches, intrinsics, M: int, b0: int = 0, b1: int | None = None,
                        gap: int = 30, radius: float = 2.0, width: float = 640.0, height: float = 480.0,
                        out: dict | None = None, sync: bool = True) -> dict:
        """Proximity loop edges for the query frames b0 <= b < b1 (see
        ba_proximity_edges): poses float64 [N,7], patches float32 [N*M,3,3,3]
        on the device; intrinsics 4 numbers (any tensor or sequence).

        ``out`` may supply the output tensors (int32 ``ii``, ``jj``, ``kk`` of
        equal length = the capacity, optional float32 [cap,2] ``coords``,
        int32 [b1-b0] ``match``, int32 [1] ``count``), e.g. views past a
        graph's local edges; missing ones are allocated with capacity
        (b1-b0)*M.  ``sync=True`` waits and returns the first n edges (n
        from the count); ``sync=False`` only queues the work (capturable)
        and returns the full buffers with the device-side count."""
        N = poses.shape[0]
        b1 = N if b1 is None else b1
        for name, t, dt in (("poses", poses, torch.float64), ("patches", patches, torch.float32)):
            if t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
                raise TypeError(f"{name}: need a contiguous CUDA {dt} tensor")
        if patches.shape[0] < N * M:
            raise ValueError("patches must hold M patches for each of the N frames")
        if isinstance(intrinsics, torch.Tensor):
            intrinsics = intrinsics.detach().cpu().tolist()
        intr = (ctypes.c_float * 4)(*[float(x) for x in intrinsics])
        Q = max(0, b1 - b0)
        dev = poses.device
        out = dict(out or {})
        if "ii" not in out:
            cap = Q * M
            for name in ("ii", "jj", "kk"):
                out[name] = torch.empty(cap, dtype=torch.int32, device=dev)
            out.setdefault("coords", torch.empty((cap, 2), dtype=torch.float32, device=dev))
        cap = out["ii"].shape[0]
        out.setdefault("match", torch.empty(max(Q, 1), dtype=torch.int32, device=dev))
        out.setdefault("count", torch.zeros(1, dtype=torch.int32, device=dev))
        for name in ("ii", "jj", "kk", "match", "count"):
            t = out[name]
            if t.dtype != torch.int32 or not t.is_contiguous() or not t.is_cuda:
                raise TypeError(f"{name}: need a contiguous CUDA int32 tensor")
        if out["jj"].shape[0] < cap or out["kk"].shape[0] < cap or out["match"].shape[0] < Q:
            raise ValueError("output tensors too short")
        coords = out.get("coords")
        if coords is not None and (coords.dtype != torch.float32 or not coords.is_contiguous()
                                   or coords.shape[0] < cap):
            raise TypeError("coords: need a contiguous CUDA float32 [cap,2] tensor")
        self._prox_keep = (poses, patches, out)
        n = ctypes.c_longlong(-1)
        capi.check(self._h, self._lib.ba_proximity_edges(
            self._h, N, M, _ptr(poses), _ptr(patches), intr, b0, b1, gap, ctypes.c_double(radius),
            ctypes.c_double(width), ctypes.c_double(height), _ptr(out["ii"]), _ptr(out["jj"]), _ptr(out["kk"]),
            _ptr(coords), ctypes.c_longlong(cap), _ptr(out["match"]), _ptr(out["count"]),
            ctypes.byref(n) if sync else None))
        if not sync:
            return out
        m = n.value
        res = {k: out[k][:m] for k in ("ii", "jj", "kk")}
        if coords is not None:
            res["coords"] = coords[:m]
        res["match"] = out["match"][:Q]
        res["n"] = m
        return res

    # ---------------------------------------------------------- correlation
    def patch_correlation(self, fmap, gmap, kk, jj, coords, radius: int = 3, out=None):
        """Eq. 4 correlation volume (see ba_patch_correlation): fmap float32
        [Nf,H,W,D] and gmap float32 [P,p,p,D] (channels last), kk/jj int32
        [E], coords float32 [E,p,p,2] (x, y) in feature-map pixels.  Returns
        (or fills) float32 [E,p,p,2R+1,2R+1]; queued on the handle's stream."""
        for name, t, dt in (("fmap", fmap, torch.float32), ("gmap", gmap, torch.float32), ("kk", kk, torch.int32),
                            ("jj", jj, torch.int32), ("coords", coords, torch.float32)):
            if t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
                raise TypeError(f"{name}: need a contiguous CUDA {dt} tensor")
        Nf, H, W, D = fmap.shape
        P, p = gmap.shape[0], gmap.shape[1]
        E = kk.shape[0]
        if gmap.shape != (P, p, p, D) or jj.shape[0] != E or coords.shape != (E, p, p, 2):
            raise ValueError("inconsistent shapes")
        G = 2 * radius + 1
        if out is None:
            out = torch.empty((E, p, p, G, G), dtype=torch.float32, device=fmap.device)
        elif out.dtype != torch.float32 or not out.is_contiguous() or out.shape != (E, p, p, G, G):
            raise TypeError("out: need a contiguous float32 [E,p,p,2R+1,2R+1] tensor")
        self._corr_keep = (fmap, gmap, kk, jj, coords, out)
        capi.check(self._h, self._lib.ba_patch_correlation(
            self._h, Nf, H, W, D, P, p, E, _ptr(fmap), _ptr(gmap), _ptr(kk), _ptr(jj), _ptr(coords), radius,
            _ptr(out)))
        return out

    # -------------------------------------------------- pose-graph optimisation
    def pgo_lm(self, S, dS, fa, fb, loop, iters: int = 20, lambda0: float = 1e-4, fd_step: float = 1e-6,
               cost=None, accepted=None):
        """Sim(3) pose-graph Levenberg-Marquardt (see ba_pgo_lm): S float64
        [N,8] (t, q xyzw, s), updated in place; dS float64 [F,8]; fa/fb/loop
        int32 [F].  Returns (cost float64 [iters+1], accepted int32 [iters]),
        queued on the handle's stream."""
        for name, t, dt in (("S", S, torch.float64), ("dS", dS, torch.float64), ("fa", fa, torch.int32),
                            ("fb", fb, torch.int32), ("loop", loop, torch.int32)):
            if t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
                raise TypeError(f"{name}: need a contiguous CUDA {dt} tensor")
        N, F = S.shape[0], fa.shape[0]
        if S.shape != (N, 8) or dS.shape != (F, 8) or fb.shape[0] != F or loop.shape[0] != F:
            raise ValueError("inconsistent shapes")
        if cost is None:
            cost = torch.empty(iters + 1, dtype=torch.float64, device=S.device)
        if accepted is None:
            accepted = torch.empty(max(iters, 1), dtype=torch.int32, device=S.device)
        if cost.dtype != torch.float64 or cost.numel() < iters + 1 or accepted.dtype != torch.int32 \
                or accepted.numel() < iters:
            raise TypeError("cost: float64 [iters+1], accepted: int32 [iters]")
        self._pgo_keep = (S, dS, fa, fb, loop, cost, accepted)
        capi.check(self._h, self._lib.ba_pgo_lm(self._h, N, F, _ptr(S), _ptr(dS), _ptr(fa), _ptr(fb), _ptr(loop),
                                                iters, lambda0, fd_step, _ptr(cost), _ptr(accepted)))
        return cost, accepted[:iters]

    # ------------------------------------------------------------ inspection
    def linearize(self, fixed: int):
        capi.check(self._h, self._lib.ba_linearize(self._h, fixed))

    def info(self) -> dict:
        arr = (ctypes.c_longlong * 16)()
        capi.check(self._h, self._lib.ba_debug_info(self._h, arr, 16))
        keys = ("N", "P", "E", "G", "groups", "n", "tile", "runs", "launches", "graph_captures", "graph_replays",
                "graph_kernels", "bind_captures", "bind_replays", "bind_kernels", "dense")
        return dict(zip(keys, list(arr)))

    def export(self, what: int, count: int | None = None) -> torch.Tensor:
        inf = self.info()
        dev = self._keep[0].device
        if what == capi.EXPORT_S:
            out = torch.empty((inf["n"], inf["n"]), dtype=torch.float64, device=dev)
        else:
            if count is None:
                count = {capi.EXPORT_Y: inf["n"], capi.EXPORT_DX: inf["n"], capi.EXPORT_DD: inf["P"],
                         capi.EXPORT_CT: inf["P"], capi.EXPORT_W: inf["P"], capi.EXPORT_PERM: inf["E"],
                         capi.EXPORT_SLOTS: inf["E"], capi.EXPORT_GPTR: inf["groups"] + 1,
                         capi.EXPORT_WIN: inf["groups"] * capi.WMAX, capi.EXPORT_COST: 1,
                         capi.EXPORT_PMPOS: inf["E"], capi.EXPORT_PPTR: inf["P"] + 1}[what]
            out = torch.empty(max(count, 1), dtype=_EXPORT_DTYPES[what], device=dev)
        capi.check(self._h, self._lib.ba_debug_export(self._h, what, _ptr(out),
                                                       out.numel() * out.element_size()))
        return out

    def profile(self, on: bool = True, classes=None):
        """Event records around every kernel class (on), none (off), or only
        the named classes (`classes`: names from capi.KERNEL_CLASSES)."""
        if classes is None:
            capi.check(self._h, self._lib.ba_profile_enable(self._h, 1 if on else 0))
            return
        mask = 0
        for name in classes:
            mask |= 1 << capi.KERNEL_CLASSES.index(name)
        capi.check(self._h, self._lib.ba_profile_classes(self._h, mask if on else 0))

    def profile_read(self) -> dict:
        """{kernel class: (total event ms, launches)} since profiling was enabled."""
        out = {}
        for k, name in enumerate(capi.KERNEL_CLASSES):
            t, n = ctypes.c_double(), ctypes.c_longlong()
            capi.check(self._h, self._lib.ba_profile_read(self._h, k, ctypes.byref(t), ctypes.byref(n)))
            out[name] = (t.value, n.value)
        return out

    def envelope(self) -> list:
        """Row envelope of each pose system above 256 unknowns as the last
        factorisation found it (ba_debug_envelope): one int32 numpy array per
        system, env[a] = first 64-column tile holding a nonzero in tile row a."""
        import numpy as np
        n = ctypes.c_longlong()
        st = self._lib.ba_debug_envelope(self._h, None, 0, ctypes.byref(n))
        if st not in (capi.BA_OK, capi.BA_ERR_INVALID_ARG):
            capi.check(self._h, st)
        buf = (ctypes.c_int * n.value)()
        capi.check(self._h, self._lib.ba_debug_envelope(self._h, buf, n.value, ctypes.byref(n)))
        v = np.frombuffer(buf, dtype=np.int32).copy()
        out, w = [], 1
        for _ in range(int(v[0])):
            T = int(v[w])
            out.append(v[w + 1:w + 1 + T])
            w += 1 + T
        return out

    def block_keys(self, fixed: int, cap: int | None = None) -> torch.Tensor:
        cap = 3 * self.E + 1 if cap is None else cap
        out = torch.empty((cap, 2), dtype=torch.int32, device=self._keep[0].device)
        n = ctypes.c_int()
        capi.check(self._h, self._lib.ba_debug_keys(self._h, fixed, _ptr(out), cap, ctypes.byref(n)))
        return out[:n.value]


class BAFunction(torch.autograd.Function):
    """The bundle adjustment as a differentiable layer: ``iters`` Gauss-Newton
    iterations from (poses, patches) with the given targets and weights,
    returning the final poses (float64 [N,7]) and inverse depths (float32 [P]).
    Gradients flow to ``targets`` and ``weights`` (the update operator's
    outputs); the initial poses and patches are treated as constants."""

    @staticmethod
    def forward(ctx, targets, weights, poses, patches, ii, jj, kk, intrinsics, iters, fixed, opts):
        targets = targets.detach().contiguous()
        weights = weights.detach().contiguous()
        T = poses.detach().clone().contiguous()
        Pt = patches.detach().clone().contiguous()
        ba = DPVBA(**(opts or {}))
        ba.set_graph(T, Pt, ii.contiguous(), jj.contiguous(), kk.contiguous(), targets, weights,
                     intrinsics.contiguous())
        ba.set_record(True)
        ba.step(iters, fixed)
        ba.sync()
        ctx.ba = ba
        ctx.target_shape = targets.shape  # [E,2], or [E,9,2] / [E,3,3,2] with residual_pixels=9
        return T, Pt[:, 2, 1, 1].clone()

    @staticmethod
    def backward(ctx, grad_poses, grad_depths):
        ba = ctx.ba
        gT, gW = ba.backward(grad_poses, grad_depths)
        ba.sync()
        return gT.reshape(ctx.target_shape), gW, None, None, None, None, None, None, None, None, None


class BAFunctionBatched(torch.autograd.Function):
    """``BAFunction`` over many independent problems bound to one handle
    (``set_graph_batched``: one launch of each kernel over all problems), e.g.
    a training batch of odometry windows.  The tensors are the problems'
    arrays concatenated (ii, jj, kk local to each problem, intrinsics [B,4]),
    ``offsets`` = (frame_off, patch_off, edge_off), each of length B+1.
    Returns the final poses [sum N,7] and inverse depths [sum P]; gradients
    flow to ``targets`` and ``weights``."""

    @staticmethod
    def forward(ctx, targets, weights, poses, patches, ii, jj, kk, intrinsics, offsets, iters, fixed, opts):
        targets = targets.detach().contiguous()
        weights = weights.detach().contiguous()
        T = poses.detach().clone().contiguous()
        Pt = patches.detach().clone().contiguous()
        ba = DPVBA(**(opts or {}))
        frame_off, patch_off, edge_off = offsets
        ba.set_graph_batched(T, Pt, ii.contiguous(), jj.contiguous(), kk.contiguous(), targets, weights,
                             intrinsics.contiguous(), frame_off, patch_off, edge_off)
        ba.set_record(True)
        ba.step(iters, fixed)
        ba.sync()
        ctx.ba = ba
        ctx.target_shape = targets.shape
        return T, Pt[:, 2, 1, 1].clone()

    @staticmethod
    def backward(ctx, grad_poses, grad_depths):
        ba = ctx.ba
        gT, gW = ba.backward(grad_poses, grad_depths)
        ba.sync()
        return gT.reshape(ctx.target_shape), gW, None, None, None, None, None, None, None, None, None, None


def bundle_adjust(targets, weights, poses, patches, ii, jj, kk, intrinsics, iters, fixed, **opts):
    """Functional form of ``BAFunction`` (keyword options as for ``DPVBA``)."""
    return BAFunction.apply(targets, weights, poses, patches, ii, jj, kk, intrinsics, iters, fixed, opts)


def bundle_adjust_batched(targets, weights, poses, patches, ii, jj, kk, intrinsics, frame_off, patch_off, edge_off,
                          iters, fixed, **opts):
    """Functional form of ``BAFunctionBatched``."""
    return BAFunctionBatched.apply(targets, weights, poses, patches, ii, jj, kk, intrinsics,
                                   (frame_off, patch_off, edge_off), iters, fixed, opts)


def batch_tensors(scene_list, device="cuda") -> tuple[dict, dict]:
    """Device copies of independent scenes concatenated for set_graph_batched:
    (tensors, offsets) with offsets frame_off / patch_off / edge_off (int64 [B+1])."""
    T = [scene_tensors(sc, device) for sc in scene_list]
    cat = {k: torch.cat([t[k] for t in T]).contiguous() for k in ("poses", "patches", "ii", "jj", "kk", "targets",
                                                                  "weights")}
    cat["intrinsics"] = torch.stack([t["intrinsics"] for t in T]).contiguous()
    offs = {name: np.r_[0, np.cumsum([getattr(sc, attr) for sc in scene_list])].astype(np.int64)
            for name, attr in (("frame_off", "N"), ("patch_off", "P"), ("edge_off", "E"))}
    return cat, offs


def scene_tensors(scene, device="cuda") -> dict:
    """Device copies of a synthetic scene's arrays in the library's layout."""
    def t(a, dt):
        return torch.as_tensor(a).to(device=device, dtype=dt).contiguous()
    return {
        "poses": t(scene.poses, torch.float64), "patches": t(scene.patches, torch.float32),
        "ii": t(scene.ii, torch.int32), "jj": t(scene.jj, torch.int32), "kk": t(scene.kk, torch.int32),
        "targets": t(scene.targets, torch.float32), "weights": t(scene.weights, torch.float32),
        "intrinsics": t(scene.intrinsics, torch.float32),
    }


def solve(scene, iters=None, fixed=None, device="cuda", **opts):
    """Bind a scene, run `iters` GN iterations, return (poses, patches) tensors."""
    T = scene_tensors(scene, device)
    ba = DPVBA(**opts)
    ba.set_graph(**T)
    ba.step(scene.iters if iters is None else iters, scene.fixed if fixed is None else fixed)
    ba.sync()
    return T["poses"], T["patches"], ba
