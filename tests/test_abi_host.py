"""CPU tests of the C-ABI library: symbols, argument checks and the host-side setup.

No GPU is touched: models are built with KT_HOST_ONLY (no device upload) and
compared with the oracle's spectrum and kept multiplets.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle.oracle import Model, Params
from paper_0908_0681_gb300 import kt, workloads

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "kt.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kt_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = kt.load()
    names = declared_functions()
    assert set(names) == set(kt.ABI_FUNCTIONS)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings():
    for code in range(9):
        assert kt.kt_status_string(code) != "unknown status"
    assert kt.kt_status_string(99) == "unknown status"


def test_rejects_bad_parameters():
    with pytest.raises(kt.KtError) as e:
        kt.kt_model_create(8, 4.0, 1.0, 1.0, 10.0, flags=kt.KT_HOST_ONLY)
    assert e.value.code == kt.KT_EINVAL
    with pytest.raises(kt.KtError):
        kt.kt_model_create(3, 4.0, 1.0, 1.0, -1.0, flags=kt.KT_HOST_ONLY)
    with pytest.raises(kt.KtError):
        kt.kt_model_create(3, 4.0, 1.0, 1.0, 1.0, precision=7, flags=kt.KT_HOST_ONLY)


def host_model(spec, flags=0, trunc_eps=None):
    return kt.kt_model_create(spec.n_orb, spec.U, spec.J, spec.mu, spec.beta, delta=spec.delta, Up=spec.up,
                              trunc_eps=spec.trunc_eps if trunc_eps is None else trunc_eps, deg_tol=spec.deg_tol,
                              krylov_tol=spec.krylov_tol, flags=flags | kt.KT_HOST_ONLY)


def oracle_model(spec, trunc_eps=None, density_only=False):
    return Model(Params(spec.n_orb, spec.U, spec.J, Up=spec.up, mu=spec.mu, delta=spec.delta, beta=spec.beta,
                        trunc_eps=spec.trunc_eps if trunc_eps is None else trunc_eps, deg_tol=spec.deg_tol,
                        density_only=density_only))


@pytest.mark.parametrize("name", ["three_orbital", "five_orbital"])
@pytest.mark.parametrize("flags", [0, kt.KT_SECTOR_BLOCKS, kt.KT_DENSITY_ONLY])
def test_host_spectrum_and_kept_set_match_oracle(name, flags):
    spec = workloads.WORKLOADS[name]().model
    m = host_model(spec, flags)
    o = oracle_model(spec, density_only=bool(flags & kt.KT_DENSITY_ONLY))
    info = kt.kt_model_query(m)
    assert info["n_states"] == 4 ** spec.n_orb
    np.testing.assert_allclose(kt.kt_model_spectrum(m), o.spectrum(), atol=1e-10)
    assert abs(info["E0"] - o.E0) < 1e-10
    kept = kt.kt_model_kept(m)
    assert info["n_kept"] == o.nkept
    np.testing.assert_allclose(np.sort(kept["e_minus_e0"]), np.sort(o.kept_E - o.E0), atol=1e-10)
    # kept blocks: (n_up, n_dn) agree with the oracle's kept sectors as a multiset
    n1 = spec.n_orb + 1
    ours = sorted(zip(kept["n_up"].tolist(), kept["n_dn"].tolist()))
    theirs = sorted((int(s) // n1, int(s) % n1) for s in o.kept_sec)
    assert ours == theirs


def test_block_structure_counts():
    """(n_up, n_dn, singly-occupied mask) blocks: counts follow from combinatorics."""
    for n in (1, 2, 3, 5):
        m = kt.kt_model_create(n, 4.0, 1.0, 2.0, 5.0, flags=kt.KT_HOST_ONLY)
        info = kt.kt_model_query(m)
        # a block is fixed by the mask m (which orbitals are single), the number D of doubly
        # occupied among the rest, and n_up of the singles: sum over |m|=s of (n-s+1)(s+1)
        expect = sum(math.comb(n, s) * (n - s + 1) * (s + 1) for s in range(n + 1))
        assert info["n_blocks"] == expect
        ms = kt.kt_model_create(n, 4.0, 1.0, 2.0, 5.0, flags=kt.KT_HOST_ONLY | kt.KT_SECTOR_BLOCKS)
        assert kt.kt_model_query(ms)["n_blocks"] == (n + 1) ** 2
        assert kt.kt_model_query(ms)["d_max"] == math.comb(n, n // 2) ** 2


def test_ell_width_closed_form():
    """Off-diagonal entries per row of H_loc (the ELL width nnz_max): a state with s singly
    occupied orbitals, u of them spin up, e empty and D doubly occupied orbitals has u (s - u)
    spin-flip and e D pair-hopping neighbours, all distinct states. Rows with fewer entries
    than the block capacity is what the items kernels of blocks up to 16 rows rely on when they
    keep a row's column indices in registers."""
    for n in (1, 2, 3, 4, 5):
        expect = max(u * (s - u) + e * (n - s - e) for s in range(n + 1) for u in range(s + 1)
                     for e in range(n - s + 1))
        for flags in (0, kt.KT_SECTOR_BLOCKS):
            info = kt.kt_model_query(kt.kt_model_create(n, 4.0, 1.0, 2.0, 5.0, flags=kt.KT_HOST_ONLY | flags))
            assert info["nnz_max"] == expect, (n, flags)
            assert info["nnz_max"] < info["kernel_dmax"]
        dd = kt.kt_model_query(kt.kt_model_create(n, 4.0, 1.0, 2.0, 5.0,
                                                  flags=kt.KT_HOST_ONLY | kt.KT_DENSITY_ONLY))
        assert dd["nnz_max"] == 0


def test_five_orbital_paper_degeneracies_host():
    """The product's own setup reproduces N_tr = 6, 31, 25 near the level crossing (Sec. IV.C)."""
    U, J = 6.0, 1.0
    mh = (5 - 0.5) * U - 4 * 2.5 * J
    for dmu, ntr in zip([4.98, 5.0, 5.02], [6, 31, 25]):
        m = kt.kt_model_create(5, U, J, mh + dmu, 50.0, trunc_eps=1.0, flags=kt.KT_HOST_ONLY)
        assert kt.kt_model_query(m)["n_kept"] == ntr


def test_trace_on_host_only_model_is_rejected():
    m = kt.kt_model_create(2, 4.0, 1.0, 2.0, 5.0, flags=kt.KT_HOST_ONLY)
    b = kt.kt_seq_batch(0, None, None, None, None)
    code = kt.load().kt_trace(m.handle, ctypes.byref(b), 1, 1, 1, None, None, 0, None)
    assert code == kt.KT_EINVAL


def test_workspace_size_grows_with_walkers():
    m = kt.kt_model_create(3, 4.0, 1.0, 5.0, 10.0, flags=kt.KT_HOST_ONLY)
    a, b = kt.kt_workspace_size(m, 10), kt.kt_workspace_size(m, 1000)
    assert 0 < a < b


def test_entry_points_reject_bad_arguments_without_touching_a_device():
    """Every documented argument check that comes before any CUDA call: null handles and
    outputs, host-only models, out-of-range sizes and shapes return KT_EINVAL; destroying a
    null handle is a no-op."""
    lib = kt.load()
    NULL = None
    i32 = ctypes.c_int32

    def call(name, *args):
        return getattr(lib, name)(*args)

    m = kt.kt_model_create(2, 4.0, 1.0, 2.0, 5.0, flags=kt.KT_HOST_ONLY)
    mh = m.handle
    b = kt.kt_seq_batch(1, None, None, None, None)
    mv = kt.kt_move_batch(None, None, None, None, None)
    out = ctypes.c_void_p()
    bad = kt.KT_EINVAL
    # traces and ratios on a host-only model
    assert call("kt_trace_ratio", mh, ctypes.byref(b), NULL, NULL, ctypes.byref(mv), NULL, NULL, NULL, NULL, NULL,
                ctypes.c_size_t(0), NULL) == bad
    assert call("kt_trace_ratio_static", mh, ctypes.byref(b), NULL, NULL, ctypes.byref(mv), NULL, NULL, NULL, NULL,
                NULL) == bad
    assert call("kt_measure", mh, ctypes.byref(b), NULL, NULL, NULL, NULL, NULL, NULL, ctypes.c_size_t(0), NULL) == bad
    assert call("kt_autotune", mh, ctypes.byref(b), NULL, NULL, NULL, NULL, ctypes.c_size_t(0), NULL,
                ctypes.byref(i32())) == bad
    assert call("kt_timing_begin", mh, i32(4)) == bad
    assert call("kt_timing_end", NULL, NULL, NULL) == bad
    assert call("kt_model_set_tiling", mh, i32(3)) == bad
    assert call("kt_model_query", NULL, NULL) == bad
    assert call("kt_workspace_size", mh, i32(-1), ctypes.byref(ctypes.c_size_t())) == bad
    assert call("kt_measure_workspace_size", mh, i32(-1), ctypes.byref(ctypes.c_size_t())) == bad
    # partial-state cache
    assert call("kt_ratio_cache_create", mh, i32(4), i32(16), ctypes.byref(out)) == bad
    assert call("kt_ratio_cache_create", NULL, i32(4), i32(16), ctypes.byref(out)) == bad
    assert call("kt_ratio_cache_create", mh, i32(0), i32(16), ctypes.byref(out)) == bad
    assert call("kt_ratio_cache_create", mh, i32(4), i32(0), ctypes.byref(out)) == bad
    assert call("kt_ratio_cache_build", NULL, ctypes.byref(b), NULL) == bad
    for name in ("kt_trace_ratio_cached", "kt_ratio_cache_propose"):
        assert call(name, NULL, ctypes.byref(b), NULL, NULL, ctypes.byref(mv), NULL, NULL, NULL, NULL, NULL) == bad
    assert call("kt_ratio_cache_commit", NULL, NULL, NULL, NULL) == bad
    call("kt_ratio_cache_destroy", NULL)
    # sweeps
    hyb = np.zeros(4 * 11)
    p = kt.kt_sweep_params(4, 8, 10, hyb.ctypes.data, 20, 0, 0)
    assert call("kt_sweep_create", mh, ctypes.byref(p), ctypes.byref(out)) == bad
    assert call("kt_sweep_create", NULL, ctypes.byref(p), ctypes.byref(out)) == bad
    assert call("kt_sweep_run", NULL, i32(1), NULL, i32(0), NULL) == bad
    assert call("kt_sweep_run_da", NULL, i32(1), NULL, i32(0), NULL) == bad
    assert call("kt_sweep_run_da_multi", NULL, i32(1), i32(4), NULL, i32(0), NULL) == bad
    sz = ctypes.c_size_t()
    assert call("kt_sweep_memory_bytes", NULL, ctypes.byref(p), i32(0), ctypes.byref(sz)) == bad
    assert call("kt_sweep_memory_bytes", mh, NULL, i32(0), ctypes.byref(sz)) == bad
    assert call("kt_sweep_collect", NULL, i32(1), NULL, NULL, NULL, NULL, i32(0), NULL) == bad
    assert call("kt_sweep_set_configs", NULL, NULL) == bad
    assert call("kt_sweep_set_stats", NULL, NULL) == bad
    assert call("kt_sweep_set_surrogate", NULL, NULL) == bad
    assert call("kt_sweep_get_state", NULL, NULL, NULL) == bad
    assert call("kt_sweep_get_accumulators", NULL, NULL, NULL) == bad
    assert call("kt_sweep_counters", NULL, NULL) == bad
    assert call("kt_sweep_reset_accumulators", NULL, NULL) == bad
    assert call("kt_sweep_feature_size", NULL, NULL) == bad
    call("kt_sweep_destroy", NULL)
    # surrogate network and the tensor-core product: shapes must be multiples of 16
    assert call("kt_mlp_create", i32(16), i32(8), ctypes.byref(out)) == bad
    assert call("kt_mlp_create", i32(15), i32(16), ctypes.byref(out)) == bad
    assert call("kt_mlp_create", i32(16), i32(16), NULL) == bad
    assert call("kt_mlp_num_params", NULL, NULL) == bad
    assert call("kt_mlp_set_params", NULL, NULL) == bad
    assert call("kt_mlp_get_params", NULL, NULL) == bad
    assert call("kt_mlp_get_grads", NULL, NULL) == bad
    assert call("kt_mlp_forward", NULL, NULL, i32(16), NULL, NULL) == bad
    assert call("kt_mlp_backward", NULL, NULL, NULL, i32(16), NULL, NULL) == bad
    assert call("kt_mlp_adam", NULL, ctypes.c_float(1e-3), NULL) == bad
    assert call("kt_mlp_error", NULL, NULL) == bad
    assert call("kt_mlp_get_tape", NULL, i32(16), NULL, NULL, NULL, NULL, NULL, NULL, NULL) == bad
    call("kt_mlp_destroy", NULL)
    assert call("kt_sweep_refresh", NULL, NULL, NULL) == bad
    A = np.zeros(64, np.uint16)
    C = np.zeros(64, np.float32)
    err = i32()
    for M_, N_, K_ in ((0, 16, 16), (1, 8, 16), (1, 16, 8), (1, 24, 16)):
        assert call("kt_gemm_bf16", ctypes.c_void_p(A.ctypes.data), i32(16), ctypes.c_void_p(A.ctypes.data), i32(16),
                    ctypes.c_void_p(C.ctypes.data), i32(16), i32(M_), i32(N_), i32(K_), ctypes.byref(err), NULL) == bad
    call("kt_model_destroy", NULL)


def test_sweep_memory_bytes_on_host_only_model():
    """kt_sweep_memory_bytes needs no device: it grows with k_cap (the inverse bath matrices,
    8 k_cap^2 bytes per flavor and walker), the partial-state cache adds the documented
    4 n_walkers n_kept (cache_ops + 1) (d_max element + 20) bytes, multi-try slots grow with
    the tries, and parameters kt_sweep_create rejects are rejected."""
    from paper_0908_0681_gb300 import engine, workloads
    spec = workloads.five_orbital_sweep().model
    m = engine.model_from_spec(spec, flags=kt.KT_HOST_ONLY)
    info = kt.kt_model_query(m)
    nw, nf = 256, info["n_flavors"]
    b64, b128 = kt.kt_sweep_memory_bytes(m, nw, 64), kt.kt_sweep_memory_bytes(m, nw, 128)
    grow = b128 - b64
    want = nw * nf * 8 * (128 ** 2 - 64 ** 2)
    assert want <= grow <= want * 1.1, (grow, want)
    P = 100
    dc = kt.kt_sweep_memory_bytes(m, nw, 64, cache_ops=P) - b64
    cache = 4 * nw * info["n_kept"] * (P + 1) * (info["d_max"] * 4 + 20)
    assert cache <= dc <= cache + 64 * 1024, (dc, cache)
    t4, t8 = (kt.kt_sweep_memory_bytes(m, nw, 64, tries=t) for t in (4, 8))
    assert b64 < t4 < t8
    with pytest.raises(RuntimeError):
        kt.kt_sweep_memory_bytes(m, nw, 129)
    with pytest.raises(RuntimeError):
        kt.kt_sweep_memory_bytes(m, nw, 64, tries=kt.KT_DA_MAX_TRIES + 1)
    assert engine.largest_cache_ops(m, nw, b64 - 1) == -1
    assert engine.largest_cache_ops(m, nw, b64) == 0
    c = engine.largest_cache_ops(m, nw, b64 + dc)
    assert c >= P and kt.kt_sweep_memory_bytes(m, nw, 64, cache_ops=c) <= b64 + dc
