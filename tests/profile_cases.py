"""Small, self-checking launch cases for profiling one kernel at a time
(test infrastructure, like the oracle it checks against).

    python tests/profile_cases.py stream --rows 8192 --cols 32768 --reps 3
    python tests/profile_cases.py gemm   --rows 8192 --cols 32768 --batch 256 --reps 2
    python tests/profile_cases.py hint   --rows 8192 --cols 32768 --n 1024 --reps 1
    python tests/profile_cases.py qbatch --cols 32768 --n 1024 --batch 1024 --client 1

Each case builds one database of the given size on cuda:0 (uniform digits,
seed 1), runs the chosen entry point `reps` times after one warm-up call,
prints the CUDA-event time per call and the bytes/flops it implies, and
checks sampled outputs against the CPU oracle so a profile is never taken of
a wrong kernel.  Sizes default to inputs larger than L2 (129 MB) with a few
GB on the device at most.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_2510_03631_gb300 import inputs, pir  # noqa: E402


def _row_check(D_row: np.ndarray, X: np.ndarray, got: np.ndarray):
    """One database row against every vector of X (B x C): the oracle's batched Response."""
    exp = oracle.answer_batch(D_row[None, :], X, threads=oracle.max_threads())[:, 0]
    if not np.array_equal(exp, got):
        raise SystemExit("profile case: output row differs from the oracle")


def _chor_case(a):
    """Chor GF(2) Response: rows x bits database, a batch of uniformly random queries."""
    rows, bits, B = a.rows, a.bits, a.batch
    W = bits // 32
    DB_np = inputs.chor_db(rows, bits, seed=1)
    Q_np = inputs.chor_queries(B, rows, seed=2)
    h = pir.qpadl_chor_setup(rows, bits, torch.from_numpy(DB_np.view(np.int32).reshape(-1)).cuda())
    if a.m4rm >= 0:
        pir.qpadl_chor_set_option(h, pir.QPADL_CHOR_OPT_M4RM_MIN_BATCH, a.m4rm)
    if a.form >= 0:
        pir.qpadl_chor_set_option(h, pir.QPADL_CHOR_OPT_SCAN_FORM, a.form)
    Q = torch.from_numpy(Q_np.view(np.int32).reshape(-1)).cuda()
    out = torch.empty(B * W, dtype=torch.int32, device="cuda")
    fn = lambda: pir.qpadl_chor_answer_batch(h, Q, out)
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    if pir.qpadl_chor_status(h) != 0:
        raise SystemExit("profile case: device status word set")
    # query 0 on the first 64 words against the oracle
    exp = oracle.chor_answer(np.ascontiguousarray(DB_np[:, :64]), rows, Q_np[:1], threads=oracle.max_threads())[0]
    if not np.array_equal(pir.as_u32(out)[:64], exp):
        raise SystemExit("profile case: output differs from the oracle")
    ms = min(times)
    alg = rows * W * 4 + B * ((rows + 31) // 32) * 4 + B * W * 4
    print(json.dumps({"case": "chor", "rows": rows, "bits": bits, "batch": B, "ms": times, "alg_bytes": alg,
                      "m4rm_min_batch": pir.qpadl_chor_get_option(h, pir.QPADL_CHOR_OPT_M4RM_MIN_BATCH),
                      "gbs": alg / (ms * 1e-3) / 1e9, "queries_per_s": B / (ms * 1e-3),
                      "db_scan_gbs": B * rows * W * 4 / (ms * 1e-3) / 1e9}))
    h.close()


def _goldberg_case(a):
    """Goldberg Response over Z_257 on a rows x cols byte database, a batch of uniform field elements."""
    R, C, B, p = a.rows, a.cols, a.batch, 257
    D_np = inputs.db_digits(R, C, 256, seed=1)
    h = pir.qpadl_goldberg_setup(R, C, p, torch.from_numpy(D_np).cuda())
    if a.pair >= 0:
        pir.qpadl_goldberg_set_option(h, pir.QPADL_GOLDBERG_OPT_PAIR_GEMM, a.pair)
    Q_np = (inputs.uniform_u32(B * C, seed=2, tag=inputs.TAG_MISC) % p).reshape(B, C)
    Q = pir.from_u32(Q_np.reshape(-1))
    out = torch.empty(B * R, dtype=torch.int32, device="cuda")
    fn = lambda: pir.qpadl_goldberg_answer_batch(h, Q, out)
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    if pir.qpadl_goldberg_status(h) != 0:
        raise SystemExit("profile case: device status word set")
    exp = oracle.goldberg_answer(D_np[R // 2][None, :], Q_np, p, threads=oracle.max_threads())[:, 0]
    if not np.array_equal(pir.as_u32(out).reshape(B, R)[:, R // 2], exp):
        raise SystemExit("profile case: output differs from the oracle")
    ms = min(times)
    print(json.dumps({"case": "goldberg", "rows": R, "cols": C, "batch": B, "ms": times,
                      "fp16_mma_flops": 2 * R * C * B, "tflops": 2 * R * C * B / (ms * 1e-3) / 1e12,
                      "queries_per_s": B / (ms * 1e-3)}))
    h.close()


def _delta_case(a):
    """Sec. 5.3 compression: width, encoding of rows x 8192 sorted entries (blocks of E = 8192), and
    decoding of `batch` blocks taken from the encoded database; checked by host prefix sums."""
    E, C = 8192, a.rows
    n = C * E
    x_np = inputs.sorted_entries(n, seed=5, max_gap=31)
    x = torch.from_numpy(x_np.view(np.int32)).cuda()
    w = pir.qpadl_pir_delta_width(x, E)
    Rp = pir.delta_rows(E, w)
    db = torch.empty(Rp * C, dtype=torch.uint8, device="cuda")
    B = min(a.batch, C)
    blocks = torch.empty(B * Rp, dtype=torch.uint8, device="cuda")
    out = torch.empty(B * E, dtype=torch.int32, device="cuda")

    def fn():
        pir.qpadl_pir_delta_encode(x, E, w, db)
        blocks.copy_(db.view(Rp, C)[:, :B].t().reshape(-1))
        pir.qpadl_pir_delta_decode(blocks, B, E, w, out)

    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    got = pir.as_u32(out).reshape(B, E)
    if not np.array_equal(got, x_np[:B * E].reshape(B, E)):
        raise SystemExit("profile case: decoded blocks differ from the entries")
    exp_db = oracle.delta_encode(x_np[:B * E], E, w)
    if not np.array_equal(blocks.cpu().numpy().reshape(B, Rp), exp_db.T):
        raise SystemExit("profile case: encoded blocks differ from the oracle")
    print(json.dumps({"case": "delta", "blocks": C, "block_entries": E, "width": w, "rows_compressed": Rp,
                      "decoded_blocks": B, "ms": times, "entry_bytes": 4 * n, "db_bytes": Rp * C}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["stream", "gemm", "hint", "query", "recover", "qbatch", "rbatch", "chor",
                                     "goldberg", "delta"])
    ap.add_argument("--rows", type=int, default=8192)
    ap.add_argument("--cols", type=int, default=32768)
    ap.add_argument("--bits", type=int, default=262144, help="chor: bits per record")
    ap.add_argument("--m4rm", type=int, default=-1, help="chor: smallest batch on the four-Russians kernel")
    ap.add_argument("--form", type=int, default=-1, help="chor: inner-loop form of the masked-XOR scan (0..3)")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--chunk", type=int, default=0, help="streaming chunk width (0 = library default)")
    ap.add_argument("--raw", type=int, default=-1, help="1: single query packed inside the kernel")
    ap.add_argument("--u8max", type=int, default=-1, help="largest batch on the uint8-digit GEMM")
    ap.add_argument("--kstep", type=int, default=-1, help="digits per row per stage of that GEMM")
    ap.add_argument("--pair", type=int, default=-1, help="1: GEMMs on tiles over pairs of SMs, 0: single-SM tiles")
    ap.add_argument("--client", type=int, default=1, help="qbatch/rbatch: 1 = tensor-core client context, "
                                                            "0 = CUDA-core batch entry point")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    if a.case == "chor":
        return _chor_case(a)
    if a.case == "goldberg":
        return _goldberg_case(a)
    if a.case == "delta":
        return _delta_case(a)
    R, C = a.rows, a.cols
    D_np = inputs.db_digits(R, C, 256, seed=1)
    prm = pir.params(R, C, a.n, seed=1)
    db = pir.qpadl_pir_setup(prm, torch.from_numpy(D_np).cuda())
    if a.chunk:
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_STREAM_CHUNK, a.chunk)
    if a.raw >= 0:
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_STREAM_RAW, a.raw)
    if a.u8max >= 0:
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_U8_MAX_BATCH, a.u8max)
    if a.kstep >= 0:
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_U8_KSTEP, a.kstep)
    if a.pair >= 0:
        pir.qpadl_pir_set_option(db, pir.QPADL_OPT_PAIR_GEMM, a.pair)
    res = {"case": a.case, "rows": R, "cols": C, "chunk": pir.qpadl_pir_get_option(db, pir.QPADL_OPT_STREAM_CHUNK),
           "pair": a.pair}
    if a.case == "stream":
        X_np = inputs.uniform_u32(C, seed=2, tag=inputs.TAG_MISC)
        q = pir.from_u32(X_np)
        ans = torch.empty(R, dtype=torch.int32, device="cuda")
        fn = lambda: pir.qpadl_pir_answer(db, q, ans)
        out_row = lambda: pir.as_u32(ans)[R // 2:R // 2 + 1]
        X_chk = X_np[None, :]
        res["alg_bytes"] = R * C + 4 * C + 4 * R
    elif a.case == "gemm":
        B = a.batch
        X_np = inputs.uniform_u32(B * C, seed=3, tag=inputs.TAG_MISC).reshape(B, C)
        Q = pir.from_u32(X_np.reshape(-1))
        ans = torch.empty(B * R, dtype=torch.int32, device="cuda")
        fn = lambda: pir.qpadl_pir_answer_batch(db, Q, ans, path=1)
        out_row = lambda: pir.as_u32(ans).reshape(B, R)[:, R // 2]
        X_chk = X_np
        res["batch"] = B
        res["fp16_mma_flops"] = 2 * R * C * 4 * B
    elif a.case in ("query", "recover"):
        # Query over A (C x n) or Recover over H (R x n): rows of a uint32 matrix against the secret
        n = a.n
        rows = C if a.case == "query" else R
        X = torch.empty(rows * n, dtype=torch.int32, device="cuda")
        pir.qpadl_pir_gen_a(pir.params(R, rows, n, seed=3), X)
        s_np = inputs.secrets(1, n, seed=4)[0]
        s_t = pir.from_u32(s_np)
        if a.case == "query":
            e = torch.from_numpy(inputs.noise(rows, seed=5)).cuda()
            q = torch.empty(rows, dtype=torch.int32, device="cuda")
            fn = lambda: pir.qpadl_pir_query(prm, X, s_t, e, 7, q)
        else:
            ans = pir.from_u32(inputs.uniform_u32(rows, seed=6, tag=inputs.TAG_MISC))
            out = torch.empty(rows, dtype=torch.uint8, device="cuda")
            fn = lambda: pir.qpadl_pir_recover(pir.params(rows, C, n), ans, X, s_t, out)
        out_row = None
        res["alg_bytes"] = rows * n * 4 + 4 * n + 8 * rows
        res["n"] = n
    elif a.case in ("qbatch", "rbatch"):
        # B queries over A (C x n) or B recoveries over H (R x n)
        n, B = a.n, a.batch
        rows = C if a.case == "qbatch" else R
        X = torch.empty(rows * n, dtype=torch.int32, device="cuda")
        pir.qpadl_pir_gen_a(pir.params(R, rows, n, seed=3), X)
        S_np = inputs.secrets(B, n, seed=4)
        S = pir.from_u32(S_np.reshape(-1))
        cprm = pir.params(R if a.case == "rbatch" else 1, rows if a.case == "qbatch" else C, n)
        cl = None
        if a.case == "qbatch":
            E_np = inputs.noise_batch(B, rows, seed=5)
            E = torch.from_numpy(E_np.reshape(-1)).cuda()
            cols = inputs.target_columns(B, rows, seed=6)
            cols_t = torch.from_numpy(cols.astype(np.int32)).cuda()
            Q = torch.empty(B * rows, dtype=torch.int32, device="cuda")
            if a.client:
                cl = pir.qpadl_client_create(cprm, X, None, max_batch=B)
                if a.pair >= 0:
                    pir.qpadl_client_set_option(cl, pir.QPADL_CLIENT_OPT_PAIR_GEMM, a.pair)
                fn = lambda: pir.qpadl_client_query_batch(cl, S, E, cols_t, Q)
            else:
                fn = lambda: pir.qpadl_pir_query_batch(cprm, X, S, E, cols_t, Q)
            def check():
                # first query against the oracle's Query
                exp = oracle.query(pir.as_u32(X).reshape(rows, n), S_np[0], E_np[0], int(cols[0]),
                                   oracle.delta_for(256))
                return np.array_equal(pir.as_u32(Q)[:rows], exp)
        else:
            ans_np = inputs.uniform_u32(B * rows, seed=6, tag=inputs.TAG_MISC)
            ans = pir.from_u32(ans_np)
            out = torch.empty(B * rows, dtype=torch.uint8, device="cuda")
            Xr = X
            if a.client:
                A_dummy = torch.zeros(C * n, dtype=torch.int32, device="cuda")
                cl = pir.qpadl_client_create(cprm, A_dummy, Xr, max_batch=B)
                if a.pair >= 0:
                    pir.qpadl_client_set_option(cl, pir.QPADL_CLIENT_OPT_PAIR_GEMM, a.pair)
                fn = lambda: pir.qpadl_client_recover_batch(cl, ans, S, out)
            else:
                fn = lambda: pir.qpadl_pir_recover_batch(cprm, ans, Xr, S, out)
            def check():
                # first recovery against the oracle's Recover
                exp = oracle.recover(ans_np[:rows], pir.as_u32(X).reshape(rows, n), S_np[0], 256)
                return np.array_equal(out.cpu().numpy()[:rows], exp)
        out_row = None
        res.update(n=n, batch=B, client=a.client, u32_macs=rows * n * B, fp16_mma_flops=2 * rows * 4 * n * 4 * B)
    else:
        n = a.n
        A = torch.empty(C * n, dtype=torch.int32, device="cuda")
        pir.qpadl_pir_gen_a(prm, A)
        H = torch.empty(R * n, dtype=torch.int32, device="cuda")
        fn = lambda: pir.qpadl_pir_hint(db, A, H)
        out_row = lambda: pir.as_u32(H).reshape(R, n)[R // 2]
        X_chk = pir.as_u32(A).reshape(C, n).T.copy()
        res["n"] = n
        res["fp16_mma_flops"] = 2 * R * C * 4 * n
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    if pir.qpadl_pir_status(db) != 0:
        raise SystemExit("profile case: device status word set")
    if out_row is not None:
        _row_check(D_np[R // 2], X_chk, out_row())
    if a.case in ("qbatch", "rbatch"):
        if not check():
            raise SystemExit("profile case: first vector differs from the oracle")
        if cl is not None and pir.qpadl_client_status(cl) != 0:
            raise SystemExit("profile case: client status word set")
    res["ms"] = times
    ms = min(times)
    if "alg_bytes" in res:
        res["gbs"] = res["alg_bytes"] / (ms * 1e-3) / 1e9
    if "fp16_mma_flops" in res:
        res["tflops"] = res["fp16_mma_flops"] / (ms * 1e-3) / 1e12
    print(json.dumps(res))
    db.close()


if __name__ == "__main__":
    main()
