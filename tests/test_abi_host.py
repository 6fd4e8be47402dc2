"""Host-side checks of the C ABI: the library builds, loads, exports every
declared entry point, validates arguments, and its binomial checkpoint plan
matches Eq. 2.18 and the brute-force optimum.  No device compute is called."""
import os
import re

import pytest

from oracle import pipe_oracle as po

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib
    return _lib


def declared_entry_points():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(pnop_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    names = declared_entry_points()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L.lib, n), n
    assert set(names) == set(L.EXPORTS)


def test_error_strings(L):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert L.lib.pnop_error_string(code)


def test_create_rejects_bad_arguments_before_touching_the_device(L):
    import ctypes
    h = ctypes.c_void_p()
    bad = [
        L.pnop_grid(4, 16, 32, 10.0, 0.0),      # nr too small
        L.pnop_grid(32, 15, 32, 10.0, 0.0),     # odd ntheta
        L.pnop_grid(32, 16, 32, -1.0, 0.0),     # negative length
    ]
    p = L.pnop_params(2000.0, 8.0, 1.0, 0.01, 0.0, 0, 8, 0)
    for g in bad:
        assert L.lib.pnop_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(h)) == -1
        assert not h.value
    g = L.pnop_grid(32, 16, 32, 10.0, 0.0)
    for q in (L.pnop_params(-1.0, 8.0, 1.0, 0.01, 0.0, 0, 8, 0), L.pnop_params(2000.0, 8.0, 1.0, 0.0, 0.0, 0, 8, 0),
              L.pnop_params(2000.0, 8.0, 1.0, 0.01, 0.0, 7, 8, 0), L.pnop_params(2000.0, -8.0, 1.0, 0.01, 0.0, 0, 0, 0)):
        assert L.lib.pnop_create(ctypes.byref(g), ctypes.byref(q), None, ctypes.byref(h)) == -1
    # physical sizes that are not 2^a 3^b: ntheta = 10 -> 15 points
    g = L.pnop_grid(32, 10, 32, 10.0, 0.0)
    assert L.lib.pnop_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(h)) == -6


def test_revolve_plan_matches_eq_2_18_and_bruteforce(L):
    C = po.revolve_advances_dp(120, 7)
    for n in range(1, 121):
        for s in range(1, 8):
            adv, stores = L.pnop_revolve_counts(n, s)
            assert adv == C[n, s] == po.revolve_advances(n, s), (n, s)
            assert stores <= max(0, n - 1)


def test_revolve_plan_large_horizons(L):
    # workloads of the paper's size: 4000 steps / 32 slots, 19635 steps / budgets
    for n, s in ((4000, 32), (1000, 4), (1000, 8), (1000, 16), (1000, 64), (19635, 40)):
        adv, _ = L.pnop_revolve_counts(n, s)
        assert adv == po.revolve_advances(n, s)
    assert L.pnop_revolve_counts(4000, 32)[0] == 11405


def _two_level_model(N, s, k, C):
    """Forward steps of the two-level schedule by construction: the forward
    phase reaches the start of the last of k + 1 near-equal intervals, then
    each interval costs its optimal binomial recomputation (brute-force table
    C), plus the terminal step."""
    if k == 0:
        return C[N, s] + 1
    b = [i * N // (k + 1) for i in range(k + 2)]
    return b[k] + sum(C[b[i + 1] - b[i], s] for i in range(k + 1)) + 1


def test_two_level_schedule_minimises_eq_2_21(L):
    C = po.revolve_advances_dp(120, 8)
    for N, s, H, r in ((30, 2, 10, 0.0), (100, 4, 40, 0.3), (120, 8, 119, 0.0), (60, 3, 5, 2.0), (50, 8, 0, 0.0),
                       (97, 2, 96, 0.05)):
        nf, adv = L.pnop_two_level_counts(N, s, H, r)
        costs = [k * r + _two_level_model(N, s, k, C) for k in range(0, min(H, N - 1) + 1)]
        best = min(costs)
        assert abs(nf * r + adv - best) < 1e-9, (N, s, H, r)
        assert costs.index(best) == nf
        assert adv == _two_level_model(N, s, nf, C)
    # enough host slots: each state is computed once (ties go to fewer host slots)
    nf, adv = L.pnop_two_level_counts(100, 2, 99, 0.0)
    assert adv == 100 and nf >= 98
    # no host slots: the single-level schedule (Eq. 2.18 + the terminal step)
    assert L.pnop_two_level_counts(100, 4, 0, 0.0) == (0, po.revolve_advances(100, 4) + 1)


def test_new_entry_points_reject_bad_arguments_without_a_device(L):
    import ctypes
    st = L.pnop_opt_stats()
    assert L.lib.pnop_optimise(None, None, 1e-3, 1.0, 5, 1e-8, None, ctypes.byref(st)) == -1
    assert L.lib.pnop_set_host_tier(None, 4, 0.0) == -1
    assert L.lib.pnop_host_tier_stats(None, None, None, None, None) == -1
    assert L.lib.pnop_mode_energy(None, None, None) == -1
    assert L.lib.pnop_gradient_continuous(None, None, 1e-3, 1.0, None, None) == -1
    assert L.lib.pnop_set_optimiser_first_step(None, 0.5) == -1
    nf, adv = ctypes.c_int(), ctypes.c_longlong()
    for args in ((0, 2, 4, 0.0), (10, 0, 4, 0.0), (10, 2, -1, 0.0), (10, 2, 4, -1.0), (10, 2, 4, float("nan"))):
        assert L.lib.pnop_two_level_counts(*args, ctypes.byref(nf), ctypes.byref(adv)) == -1


def test_batch_entry_points_reject_bad_arguments_without_a_device(L):
    import ctypes
    g = L.pnop_grid(12, 8, 12, 6.0, 0.0)
    h = ctypes.c_void_p()
    for cap, snaps in ((0, 2), (L.PNOP_MAX_BATCH + 1, 2), (4, 0)):
        p = L.pnop_params(2000.0, 8.0, 1.0, 0.01, 0.0, 0, snaps, 0)
        assert L.lib.pnop_batch_create(ctypes.byref(g), ctypes.byref(p), cap, None, ctypes.byref(h)) == -1
        assert h.value is None
    p = L.pnop_params(2000.0, 8.0, 1.0, 0.01, 0.0, 0, 2, 0)
    assert L.lib.pnop_batch_create(None, ctypes.byref(p), 2, None, ctypes.byref(h)) == -1
    i, t = ctypes.c_int(), ctypes.c_longlong()
    assert L.lib.pnop_batch_submit(None, ctypes.byref(p), None, 1e-3, 1.0, ctypes.byref(i)) == -1
    assert L.lib.pnop_batch_run(None, 4, None, None) == -1
    assert L.lib.pnop_batch_poll(None, 0, ctypes.byref(i)) == -1
    assert L.lib.pnop_batch_result(None, 0, None, None) == -1
    assert L.lib.pnop_batch_stats(None, ctypes.byref(t), None, None) == -1
    o = ctypes.c_void_p()
    assert L.lib.pnop_batch_prepare(None, ctypes.byref(p), ctypes.byref(o)) == -1 and o.value is None
    assert L.lib.pnop_batch_submit_prepared(None, None, None, 1e-3, 1.0, ctypes.byref(i)) == -1
    L.lib.pnop_ops_free(None)
    L.lib.pnop_batch_destroy(None)


def test_batch_bytes_estimate_grows_with_capacity_and_checkpoints(L):
    b = {c: L.pnop_batch_bytes(64, 64, 256, 100.0, L.PNOP_MIXED, 8, c) for c in (1, 2, 8)}
    assert b[1] < b[2] < b[8] and b[8] > 7 * (b[2] - b[1])
    assert L.pnop_batch_bytes(64, 64, 256, 100.0, L.PNOP_MIXED, 16, 2) > b[2]
    assert L.pnop_batch_bytes(64, 64, 256, 100.0, L.PNOP_FP64, 8, 2) > b[2]
    field = 3 * 64 * 63 * 128 * 16
    assert b[2] > 2 * (18 + 8) * field  # at least the per-slot fields
    import ctypes
    g = L.pnop_grid(64, 64, 256, 100.0, 0.0)
    out = ctypes.c_size_t()
    for cap, snaps in ((0, 8), (17, 8), (2, 0)):
        p = L.pnop_params(1.0, 1.0, 0.0, 1.0, 0.0, 1, snaps, 0)
        assert L.lib.pnop_batch_bytes(ctypes.byref(g), ctypes.byref(p), cap, ctypes.byref(out)) == -1


def test_noalloc_energy_rejects_oversized_fields_without_a_device(L):
    """pnop_energy_noalloc checks 3 nr (2M+1) (K+1) against its fixed scratch
    before any CUDA call, one factor at a time, so sizes whose product would
    overflow 64 bits are rejected too.  Non-null dummy pointers are never
    dereferenced on these paths."""
    import ctypes
    dummy = ctypes.c_void_p(16)
    e = ctypes.c_double()
    INT_MAX = 2 ** 31 - 1
    cases = [
        (INT_MAX, INT_MAX // 2, INT_MAX - 1),      # product far beyond 2^63
        (INT_MAX, 0, 0),                           # first factor alone too large
        (64, 0, 87381),                            # 3*64*87382 = 2^24 + 128: one step past the limit
        (512, 127, 255),
    ]
    for nr, M, K in cases:
        rc = L.lib.pnop_energy_noalloc(dummy, ctypes.cast(dummy, ctypes.POINTER(ctypes.c_double)), nr, M, K, 10.0,
                                       ctypes.byref(e), None)
        assert rc == -1, (nr, M, K)


def test_fma_probe_rejects_bad_arguments_without_a_device(L):
    import ctypes
    t = ctypes.c_double()
    for prec, secs in ((0, 0.0), (0, -1.0), (0, 11.0), (7, 0.1)):
        assert L.lib.pnop_measure_fma_peak(prec, secs, None, ctypes.byref(t)) == -1
    assert L.lib.pnop_measure_fma_peak(0, 0.1, None, None) == -1


def test_a_plain_c_program_uses_the_abi(L, tmp_path):
    """The public header compiles as C99 with warnings as errors, and a C
    program linked against the library calls host-only entry points."""
    import shutil
    import subprocess
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_pnop.c"
    src.write_text(
        "#include <stdio.h>\n#include \"pnop.h\"\n"
        "int main(void) {\n"
        "    long long adv = 0, st = 0;\n"
        "    if (pnop_revolve_counts(100, 4, &adv, &st) != PNOP_OK) return 1;\n"
        "    if (pnop_set_optimiser_first_step((pnop_ctx*)0, 0.5) != PNOP_ERR_INVALID_ARG) return 2;\n"
        "    printf(\"%lld %lld\\n\", adv, st);\n"
        "    return 0;\n"
        "}\n")
    libdir = os.path.dirname(os.path.abspath(L.lib._name))
    exe = tmp_path / "use_pnop"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", libdir, "-lpnop", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert int(out[0]) == po.revolve_advances(100, 4)
