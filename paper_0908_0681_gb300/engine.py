"""Convenience layer over the binding: device-resident batches and one-call traces.

Moves arrays to the GPU with torch, sizes the workspace and calls the C ABI;
it computes nothing itself.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import kt


@dataclass
class DeviceSeqs:
    offsets: torch.Tensor
    tau: torch.Tensor
    flavor: torch.Tensor
    dagger: torch.Tensor

    @staticmethod
    def from_host(seqs, device="cuda") -> "DeviceSeqs":
        return DeviceSeqs(torch.as_tensor(np.asarray(seqs.offsets, np.int32), device=device),
                          torch.as_tensor(np.asarray(seqs.tau, np.float64), device=device),
                          torch.as_tensor(np.asarray(seqs.flavor, np.uint8), device=device),
                          torch.as_tensor(np.asarray(seqs.dagger, np.uint8), device=device))

    @property
    def n(self) -> int:
        return self.offsets.numel() - 1

    def batch(self) -> kt.kt_seq_batch:
        return kt.seq_batch(self.offsets, self.tau, self.flavor, self.dagger)

    def nbytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in (self.offsets, self.tau, self.flavor, self.dagger))


@dataclass
class DeviceMoves:
    kind: torch.Tensor
    flavor: torch.Tensor
    t_dag: torch.Tensor
    t_ann: torch.Tensor
    rem_idx: torch.Tensor

    @staticmethod
    def from_host(mv, device="cuda") -> "DeviceMoves":
        return DeviceMoves(torch.as_tensor(np.asarray(mv.kind, np.uint8), device=device),
                           torch.as_tensor(np.asarray(mv.flavor, np.uint8), device=device),
                           torch.as_tensor(np.asarray(mv.t_dag, np.float64), device=device),
                           torch.as_tensor(np.asarray(mv.t_ann, np.float64), device=device),
                           torch.as_tensor(np.asarray(mv.rem_idx, np.int32), device=device))

    def batch(self) -> kt.kt_move_batch:
        return kt.move_batch(self.kind, self.flavor, self.t_dag, self.t_ann, self.rem_idx)

    def nbytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in (self.kind, self.flavor, self.t_dag, self.t_ann, self.rem_idx))


def model_from_spec(spec, precision=kt.KT_FP32_KRYLOV, flags=0, krylov_pmax=0, trunc_eps=None) -> kt.KtModel:
    return kt.kt_model_create(spec.n_orb, spec.U, spec.J, spec.mu, spec.beta, delta=spec.delta,
                              Up=spec.up, trunc_eps=spec.trunc_eps if trunc_eps is None else trunc_eps,
                              deg_tol=spec.deg_tol, krylov_tol=spec.krylov_tol, krylov_pmax=krylov_pmax,
                              precision=precision, flags=flags)


def new_stats(device="cuda") -> torch.Tensor:
    return torch.zeros(kt.STATS_WORDS, dtype=torch.int64, device=device)


def workspace(model: kt.KtModel, n: int, device="cuda") -> torch.Tensor:
    return torch.empty(max(kt.kt_workspace_size(model, n), 1), dtype=torch.uint8, device=device)


def trace(model: kt.KtModel, seqs: DeviceSeqs, stats: torch.Tensor | None = None, ws: torch.Tensor | None = None):
    """(sign int8, log|T| float64, status int32) device tensors for every walker."""
    n = seqs.n
    dev = seqs.offsets.device
    sign = torch.empty(n, dtype=torch.int8, device=dev)
    la = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    ws = workspace(model, n, dev) if ws is None else ws
    kt.kt_trace(model, seqs.batch(), sign, la, st, stats, ws)
    return sign, la, st


def measure(model: kt.KtModel, seqs: DeviceSeqs, stats: torch.Tensor | None = None, ws: torch.Tensor | None = None):
    """Observables at tau = beta/2 (kt_measure): (sign, log|T|, obs [n, KT_MEASURE_NOBS], status)."""
    n = seqs.n
    dev = seqs.offsets.device
    n_orb = kt.kt_model_query(model)["n_orb"]
    sign = torch.empty(n, dtype=torch.int8, device=dev)
    la = torch.empty(n, dtype=torch.float64, device=dev)
    obs = torch.empty((n, kt.measure_nobs(n_orb)), dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    if ws is None:
        ws = torch.empty(max(kt.kt_measure_workspace_size(model, n), 1), dtype=torch.uint8, device=dev)
    kt.kt_measure(model, seqs.batch(), sign, la, obs, st, stats, ws)
    return sign, la, obs, st


def measure_layout(n_orb: int) -> dict:
    """Column slices of kt_measure's output: n_f, double occupancy, S^2, (n_up, n_dn) histogram."""
    nf = 2 * n_orb
    return {"n": slice(0, nf), "docc": slice(nf, nf + n_orb), "S2": slice(nf + n_orb, nf + n_orb + 1),
            "sector": slice(nf + n_orb + 1, nf + n_orb + 1 + (n_orb + 1) ** 2)}


def trace_ratio(model: kt.KtModel, seqs: DeviceSeqs, cur_sign: torch.Tensor, cur_logabs: torch.Tensor,
                moves: DeviceMoves, stats: torch.Tensor | None = None, ws: torch.Tensor | None = None):
    """(sign int8, log|ratio| float64, status int32) device tensors for every walker."""
    n = seqs.n
    dev = seqs.offsets.device
    sign = torch.empty(n, dtype=torch.int8, device=dev)
    lr = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    ws = workspace(model, n, dev) if ws is None else ws
    kt.kt_trace_ratio(model, seqs.batch(), cur_sign, cur_logabs, moves.batch(), sign, lr, st, stats, ws)
    return sign, lr, st


class RatioCache:
    """Partial-state cache of fixed current configurations (kt_ratio_cache_*): build it once
    for a batch, then evaluate trace ratios of updates against those configurations by
    propagating only each update's edited window."""

    def __init__(self, model: kt.KtModel, n_walkers: int, max_ops: int = 512):
        self.h = kt.KtRatioCache(model, n_walkers, max_ops)

    def build(self, seqs: DeviceSeqs) -> None:
        kt.kt_ratio_cache_build(self.h, seqs.batch())

    def ratio(self, seqs: DeviceSeqs, cur_sign: torch.Tensor, cur_logabs: torch.Tensor, moves: DeviceMoves,
              out=None, stats: torch.Tensor | None = None):
        """(sign int8, log|ratio| float64, status int32) device tensors, as trace_ratio."""
        n = seqs.n
        dev = seqs.offsets.device
        if out is None:
            out = (torch.empty(n, dtype=torch.int8, device=dev), torch.empty(n, dtype=torch.float64, device=dev),
                   torch.empty(n, dtype=torch.int32, device=dev))
        kt.kt_trace_ratio_cached(self.h, seqs.batch(), cur_sign, cur_logabs, moves.batch(), *out, stats)
        return out

    def propose(self, seqs: DeviceSeqs, cur_sign: torch.Tensor, cur_logabs: torch.Tensor, moves: DeviceMoves,
                out=None):
        """As ratio(), keeping each update's window states aside for commit()."""
        n = seqs.n
        dev = seqs.offsets.device
        if out is None:
            out = (torch.empty(n, dtype=torch.int8, device=dev), torch.empty(n, dtype=torch.float64, device=dev),
                   torch.empty(n, dtype=torch.int32, device=dev))
        kt.kt_ratio_cache_propose(self.h, seqs.batch(), cur_sign, cur_logabs, moves.batch(), *out)
        return out

    def commit(self, accepted: torch.Tensor, status: torch.Tensor) -> None:
        """accepted: int8 device tensor (nonzero = accepted); status: the propose() statuses.
        The caller then edits its sequences of the accepted walkers as the library does."""
        kt.kt_ratio_cache_commit(self.h, accepted, status)


def binning_analysis(x) -> dict:
    """Standard error of the mean of correlated measurements by binning.

    x: [n_chains, n_t] series (or [n_t] for one chain), consecutive in Monte Carlo time.
    For every bin size b dividing n_t the series is cut into bins of b consecutive values,
    and the error of the grand mean is sqrt(var(bin means) / number of bins), pooled over
    the independent chains. For uncorrelated data every b gives the same error; with
    autocorrelation the error grows with b until the bins are longer than the
    autocorrelation time, where it levels off (the plateau is the error bar). With many
    independent chains the largest bin is a whole chain, whose mean is independent of the
    others whatever the autocorrelation. Returns {"errors": {b: error}, "error": the error
    at the largest b that leaves at least 8 bins in all, "tau_int": half the squared ratio
    of that error to the b = 1 error (the integrated autocorrelation time, in
    measurements), "plateau": whether that error is within 10% of the one at the next
    smaller b (else the series is too short for a single chain's error bar)}."""
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[None, :]
    nc, nt = x.shape
    errs = {}
    for b in range(1, nt + 1):
        if nt % b:
            continue
        y = x.reshape(nc, nt // b, b).mean(axis=2).ravel()
        if y.size < 2:
            continue
        errs[b] = float(np.sqrt(y.var(ddof=1) / y.size))
    ok = [b for b in errs if nc * (nt // b) >= 8] or list(errs)
    bmax = max(ok)
    e1 = errs[min(errs)]
    smaller = [b for b in errs if b < bmax]
    plateau = bool(smaller) and errs[bmax] <= 1.1 * errs[max(smaller)]
    return {"errors": errs, "error": errs[bmax], "tau_int": 0.5 * (errs[bmax] / e1) ** 2 if e1 > 0 else 0.5,
            "plateau": plateau}


class Sweep:
    """Batched CT-HYB Markov chains on the device (kt_sweep_*): Metropolis insertion and
    removal of c^+/c pairs with FP64 determinant updates and the library's trace ratios."""

    def __init__(self, model: kt.KtModel, hyb: np.ndarray, beta: float, n_walkers: int, k_cap: int = 64,
                 n_bins: int = 100, measure_obs: bool = False, cache_ops: int = 0):
        """cache_ops > 0 keeps the partial-state cache for walkers of up to cache_ops
        operators: each proposal's trace ratio then propagates only the stretch around its
        edit that the cache does not cover."""
        self.h = kt.KtSweep(model, hyb, n_walkers, k_cap=k_cap, n_bins=n_bins, measure_obs=measure_obs,
                            cache_ops=cache_ops)
        info = kt.kt_model_query(model)
        self.nf, self.n_orb = info["n_flavors"], info["n_orb"]
        self.beta = float(beta)
        self.n_walkers, self.k_cap, self.n_bins = int(n_walkers), int(k_cap), int(n_bins)
        self.capacity = 2 * self.nf * self.k_cap

    def run(self, uniforms: torch.Tensor, meas_every: int = 0) -> None:
        """uniforms: float64 device tensor [n_steps, n_walkers, 6]."""
        assert uniforms.dtype == torch.float64 and uniforms.is_cuda and uniforms.is_contiguous()
        assert uniforms.shape[1:] == (self.n_walkers, 6)
        kt.kt_sweep_run(self.h, uniforms.shape[0], uniforms, meas_every)

    def set_configs(self, seqs) -> None:
        """Start every chain from the given configurations (a Sequences-like CSR batch on the host)."""
        kt.kt_sweep_set_configs(self.h, seqs.offsets, seqs.tau, seqs.flavor, seqs.dagger)

    def state(self) -> dict:
        nw, cap, dev = self.n_walkers, self.capacity, "cuda"
        out = {"lens": torch.empty(nw, dtype=torch.int32, device=dev),
               "tau": torch.empty((nw, cap), dtype=torch.float64, device=dev),
               "flavor": torch.empty((nw, cap), dtype=torch.uint8, device=dev),
               "dagger": torch.empty((nw, cap), dtype=torch.uint8, device=dev),
               "sign": torch.empty(nw, dtype=torch.int8, device=dev),
               "trace_sign": torch.empty(nw, dtype=torch.int8, device=dev),
               "trace_logabs": torch.empty(nw, dtype=torch.float64, device=dev),
               "det_logabs": torch.empty(nw, dtype=torch.float64, device=dev),
               "order": torch.empty((nw, self.nf), dtype=torch.int32, device=dev)}
        kt.kt_sweep_get_state(self.h, **out)
        return out

    def configs(self) -> list:
        """Current configurations as host lists of (tau, flavor, dagger)."""
        st = {k: v.cpu().numpy() for k, v in self.state().items()}
        res = []
        for w in range(self.n_walkers):
            k = int(st["lens"][w])
            res.append(list(zip(st["tau"][w, :k].tolist(), st["flavor"][w, :k].tolist(), st["dagger"][w, :k].tolist())))
        return res

    def accumulators(self) -> dict:
        nw, dev = self.n_walkers, "cuda"
        out = {"g_tau": torch.zeros((nw, self.nf, self.n_bins), dtype=torch.float64, device=dev),
               "sign_sum": torch.zeros(nw, dtype=torch.float64, device=dev),
               "order_sum": torch.zeros((nw, self.nf), dtype=torch.float64, device=dev),
               "obs_sum": torch.zeros((nw, kt.measure_nobs(self.n_orb)), dtype=torch.float64, device=dev)}
        kt.kt_sweep_get_accumulators(self.h, **out)
        return out

    def counters(self) -> dict:
        return kt.kt_sweep_counters(self.h)

    @property
    def n_features(self) -> int:
        return kt.kt_sweep_feature_size(self.h)

    def collect(self, uniforms: torch.Tensor, capacity: int):
        """Plain steps that record (features, log|T_new/T_old|) of every evaluated nonzero ratio.
        Returns (features bf16 [n, n_in], targets float32 [n]) with n = min(count, capacity)."""
        assert uniforms.dtype == torch.float64 and uniforms.is_cuda and uniforms.is_contiguous()
        assert uniforms.shape[1:] == (self.n_walkers, 6)
        feats = torch.empty((capacity, self.n_features), dtype=torch.bfloat16, device="cuda")
        targs = torch.empty(capacity, dtype=torch.float32, device="cuda")
        count = torch.zeros(1, dtype=torch.int32, device="cuda")
        kt.kt_sweep_collect(self.h, uniforms.shape[0], uniforms, feats, targs, count)
        n = min(int(count.item()), capacity)
        return feats[:n], targs[:n]

    def set_surrogate(self, net) -> None:
        kt.kt_sweep_set_surrogate(self.h, None if net is None else net.h)

    def run_da(self, uniforms: torch.Tensor, meas_every: int = 0) -> None:
        """Delayed-acceptance steps; uniforms float64 [n_steps, n_walkers, 7]."""
        assert uniforms.dtype == torch.float64 and uniforms.is_cuda and uniforms.is_contiguous()
        assert uniforms.shape[1:] == (self.n_walkers, 7)
        kt.kt_sweep_run_da(self.h, uniforms.shape[0], uniforms, meas_every)

    def run_da_multi(self, uniforms: torch.Tensor, meas_every: int = 0) -> None:
        """Multi-try delayed-acceptance steps (kt_sweep_run_da_multi); uniforms float64
        [n_steps, n_walkers, tries, 7]. Each step takes 1 to `tries` Metropolis steps per
        walker; measurements are weighted by them."""
        assert uniforms.dtype == torch.float64 and uniforms.is_cuda and uniforms.is_contiguous()
        assert uniforms.dim() == 4 and uniforms.shape[1] == self.n_walkers and uniforms.shape[3] == 7
        kt.kt_sweep_run_da_multi(self.h, uniforms.shape[0], uniforms.shape[2], uniforms, meas_every)

    def refresh(self) -> dict:
        """Drift guard (kt_sweep_refresh): tracked M, determinants, signs and traces recomputed
        from scratch; returns how far the tracked values had drifted."""
        return kt.kt_sweep_refresh(self.h)

    def reset_accumulators(self) -> None:
        kt.kt_sweep_reset_accumulators(self.h)

    def set_stats(self, stats: torch.Tensor | None) -> None:
        """Accumulate the trace pipeline's kt_stats of the following steps into `stats`
        (engine.new_stats()); None stops."""
        self._stats = stats
        kt.kt_sweep_set_stats(self.h, stats)

    def run_blocks(self, uniforms: torch.Tensor, meas_every: int, n_blocks: int, delayed: bool = False) -> list:
        """Run the steps as n_blocks consecutive equal blocks (plain; delayed acceptance
        with 7 uniforms per step; multi-try delayed acceptance with [tries, 7] uniforms per
        step) and return each block's own accumulator sums (device
        tensors), for binning analyses over time. The running accumulators and counters
        keep their totals; the per-block sums are differences of device snapshots, so no
        block waits for the host."""
        n = uniforms.shape[0]
        assert n_blocks > 0 and n % n_blocks == 0 and meas_every > 0 and (n // n_blocks) % meas_every == 0
        step = n // n_blocks
        snaps = [self.accumulators()]
        for b in range(n_blocks):
            fn = (self.run_da_multi if uniforms.dim() == 4 else self.run_da) if delayed else self.run
            fn(uniforms[b * step:(b + 1) * step], meas_every)
            snaps.append(self.accumulators())
        return [{k: snaps[b + 1][k] - snaps[b][k] for k in snaps[0]} for b in range(n_blocks)]

    def green_function(self, acc: dict | None = None) -> torch.Tensor:
        """G_f(tau) at the bin centres, pooled over walkers: [n_flavors, n_bins]."""
        acc = self.accumulators() if acc is None else acc
        return acc["g_tau"].sum(0) * (self.n_bins / self.beta ** 2) / acc["sign_sum"].sum()


def largest_cache_ops(model: kt.KtModel, n_walkers: int, budget_bytes: int, k_cap: int = 64, n_tau: int = 2000,
                      n_bins: int = 100, measure_obs: bool = False, tries: int = 0) -> int:
    """The longest partial-state cache (operators per walker, up to the sequence capacity
    2 n_flavors k_cap) whose sweep fits in budget_bytes of device memory (for example a share of
    torch.cuda.mem_get_info()[0]); 0 if only the uncached sweep fits, -1 if not even that."""
    def need(c):
        return kt.kt_sweep_memory_bytes(model, n_walkers, k_cap, n_tau, n_bins, measure_obs, c, tries)
    if need(0) > budget_bytes:
        return -1
    lo, hi = 0, 2 * kt.kt_model_query(model)["n_flavors"] * k_cap
    if need(hi) <= budget_bytes:
        return hi
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if need(mid) <= budget_bytes:
            lo = mid
        else:
            hi = mid
    return lo


class Surrogate:
    """The delayed-acceptance network (kt_mlp_*): predicts log|T_new / T_old| of a proposal."""

    def __init__(self, n_in: int, max_batch: int = 4096, params: np.ndarray | None = None, seed: int = 0):
        self.h = kt.KtMlp(n_in, max_batch)
        self.n_in = n_in
        if params is None:
            rng = np.random.default_rng(seed)
            H = kt.KT_MLP_HIDDEN
            params = np.concatenate([rng.normal(0, np.sqrt(2.0 / n_in), H * n_in), np.zeros(H),
                                     rng.normal(0, np.sqrt(2.0 / H), H * H), np.zeros(H),
                                     rng.normal(0, np.sqrt(2.0 / H), H), np.zeros(1)])
        self.set_params(params)

    def set_params(self, params: np.ndarray) -> None:
        kt.kt_mlp_set_params(self.h, params)

    def params(self) -> np.ndarray:
        return kt.kt_mlp_get_params(self.h)

    def predict(self, X: torch.Tensor) -> torch.Tensor:
        """Network outputs for the rows of X (in chunks of max_batch)."""
        y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        mb = self.h.max_batch
        for i in range(0, X.shape[0], mb):
            kt.kt_mlp_forward(self.h, X[i:i + mb].contiguous(), y[i:i + mb])
        return y

    def train(self, X: torch.Tensor, t: torch.Tensor, epochs: int = 3, batch: int = 4096, lr: float = 1e-3,
              seed: int = 0) -> list:
        """Adam on the mean squared error; returns the mean loss of every epoch."""
        n = (X.shape[0] // batch) * batch
        g = torch.Generator(device=X.device).manual_seed(seed)
        loss = torch.zeros(1, dtype=torch.float32, device=X.device)
        hist = []
        for _ in range(epochs):
            perm = torch.randperm(X.shape[0], device=X.device, generator=g)[:n]
            tot = torch.zeros((), dtype=torch.float64, device=X.device)
            for i in range(0, n, batch):
                idx = perm[i:i + batch]
                kt.kt_mlp_backward(self.h, X[idx].contiguous(), t[idx].contiguous(), loss)
                kt.kt_mlp_adam(self.h, lr)
                tot += loss[0].double()
            hist.append(float(tot.item()) / max(n // batch, 1))
        if kt.kt_mlp_error(self.h):
            raise kt.KtError("a tensor-core wait timed out during training")
        return hist
