"""Measured error of every result of the CUDA path against the FP64 oracle, at the benchmarked
sizes (sampled where the oracle would take too long).  Not a pytest module: it measures, it
does not assert.  Two phases, so that the oracle's share runs on any host:

  python tests/error_table.py gpu  OUT.npz     # the CUDA path (needs a GPU); saves its outputs
  python tests/error_table.py report OUT.npz   # the oracle on the same inputs; prints a table

Workloads:
* the dense symmetric tensor n = 400, k = 20, B = 10, b = 2^14, L = 50, T = 30 (planted,
  noise 0.005): sketch (Eq. 7), per-sketch T^(I,u,u) (Eq. 14) and T^(u,u,u) (Eq. 13),
  Alg. 1's last power update, eigenvalues and components of every round, deflated sketches;
* the paper's synthetic grid cell n = 1000, B = 20, b = 2^14 (Sec. 5.1), where the power
  iterations converge: components and eigenvalues of an FP64 oracle run from the same starts;
* spectral LDA with V = 50000 words and k = 100 topics: the whitening identity W^T M2^ W = I on
  the benchmarked corpus (D = 10^6, evaluated with the device's M2^ operator, itself checked
  against the oracle in the test suite), and M3^(W,W,W) contracted with random vectors against
  the oracle's O(nnz k) contractions on a D = 2 10^4 document corpus.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)

import synth  # noqa: E402

CFG = dict(n=400, k=20, noise=0.005, B=10, log2b=14, L=50, T=30, seed=1)
LDA = dict(V=50000, k=100, D_full=1000000, D_m3=20000, alpha=0.1, beta=0.01, mean_len=200,
           oversample=10, power_iters=2, seed=1)
SAMPLE_TAUS = (0, 17, 49)
E1 = dict(n=1000, k=10, L=30, T=30, sigma=0.01, seed=7, B=20, log2b=14)


def gpu_phase(out):
    import torch
    import paper_1506_04448_gb300 as tsk
    dev = torch.device("cuda", 0)
    c = CFG
    r = {}
    T, _, A = synth.planted_symmetric(c["n"], c["k"], c["noise"], c["seed"], dtype=np.float32)
    U0 = synth.gaussian_inits(c["k"], c["L"], c["n"], c["seed"] + 1).astype(np.float32)
    h, g = tsk.cs_hashes(c["seed"], c["B"], c["log2b"], [c["n"]], dev)
    S = tsk.sketch_tensor(torch.from_numpy(T).to(dev), h, g, c["log2b"])
    res = tsk.robust_power_method(S, h, g, torch.from_numpy(U0).to(dev), c["T"],
                                  return_deflated=True, return_trace=True)
    tsk.check_status(dev)
    Ui = res["U_iters"]
    k, Tn = c["k"], c["T"]
    tau = res["tau"].long()
    rr = torch.arange(k, device=dev)
    r["S"] = S.cpu().numpy()
    r["h"] = h.cpu().numpy()[:, 0]
    r["g"] = g.cpu().numpy()[:, 0]
    r["lam"] = res["lam"].cpu().numpy()
    r["V"] = res["V"].cpu().numpy()
    r["tau"] = res["tau"].cpu().numpy()
    r["lam_all"] = res["lam_all"].cpu().numpy()
    r["S_deflated"] = res["S_deflated"].cpu().numpy()
    r["U_prev_sel"] = Ui[rr, Tn - 2, tau].cpu().numpy()     # selected vector, step T-1 input
    r["U_last_sel"] = Ui[rr, Tn - 1, tau].cpu().numpy()
    r["U_round0"] = Ui[0][:, list(SAMPLE_TAUS)].cpu().numpy()   # [T][3][n]
    # per-sketch contractions of four vectors against the input sketches
    U4 = torch.stack([Ui[0, Tn - 1, t] for t in SAMPLE_TAUS] +
                     [torch.nn.functional.normalize(torch.from_numpy(U0[0, 0]).to(dev), dim=0)])
    U4 = U4.contiguous()
    FS = tsk.sketch_fft(S)
    Vmed, Vall = tsk.contract_iuu(FS, S, h, g, U4, return_all=True)
    lmed, lall = tsk.contract_uuu(FS, S, h, g, U4, return_all=True)
    torch.cuda.synchronize(dev)
    r["U4"] = U4.cpu().numpy()
    r["iuu_all"] = Vall.cpu().numpy()
    r["iuu_med"] = Vmed.cpu().numpy()
    r["uuu_all"] = lall.cpu().numpy()
    r["uuu_med"] = lmed.cpu().numpy()
    del T
    # the paper's synthetic grid cell B = 20, b = 2^14 (n = 1000, full rank, noise 0.01 / n^1.5),
    # where Alg. 1 converges: components end to end
    e = E1
    T1, _, _ = synth.paper_synthetic(e["n"], e["sigma"], e["seed"])
    h1, g1 = tsk.cs_hashes(e["seed"], e["B"], e["log2b"], [e["n"]], dev)
    S1 = tsk.sketch_tensor(torch.from_numpy(T1).to(dev), h1, g1, e["log2b"])
    del T1
    U1 = synth.gaussian_inits(e["k"], e["L"], e["n"], e["seed"] + 3).astype(np.float32)
    res1 = tsk.robust_power_method(S1, h1, g1, torch.from_numpy(U1).to(dev), e["T"],
                                   return_deflated=True)
    tsk.check_status(dev)
    r["e1_S"] = S1.cpu().numpy()
    r["e1_lam"] = res1["lam"].cpu().numpy()
    r["e1_V"] = res1["V"].cpu().numpy()
    r["e1_tau"] = res1["tau"].cpu().numpy()
    r["e1_S_deflated"] = res1["S_deflated"].cpu().numpy()
    torch.cuda.empty_cache()
    # spectral LDA: whitening identity on the benchmarked corpus
    lc = LDA
    a0 = lc["k"] * lc["alpha"]
    for tag, D in (("full", lc["D_full"]), ("m3", lc["D_m3"])):
        cp = synth.lda_corpus(lc["V"], lc["k"], D, lc["seed"], alpha=lc["alpha"], beta=lc["beta"],
                              mean_len=lc["mean_len"])
        ip, idx, cnt = (torch.from_numpy(np.ascontiguousarray(cp[x])).to(dev)
                        for x in ("indptr", "idx", "cnt"))
        Om = torch.from_numpy(synth.gaussian_matrix(lc["V"], lc["k"] + lc["oversample"],
                                                    lc["seed"] + 1).astype(np.float32)).to(dev)
        W, sigma, _ = tsk.lda_whiten(ip, idx, cnt, lc["V"], lc["k"], a0, Om, lc["power_iters"])
        M2W = tsk.lda_m2_apply(ip, idx, cnt, lc["V"], a0, W)
        G = W.double().T @ M2W.double()
        r[f"lda_{tag}_gram"] = G.cpu().numpy()
        r[f"lda_{tag}_sigma"] = sigma.cpu().numpy()
        if tag == "m3":
            M3 = tsk.lda_whitened_m3(ip, idx, cnt, lc["V"], W, a0)
            r["lda_m3_W"] = W.cpu().numpy()
            r["lda_m3_M3"] = M3.cpu().numpy()
        tsk.check_status(dev)
        del ip, idx, cnt, cp
        torch.cuda.empty_cache()
    np.savez_compressed(out, **r)
    print("saved", out)


def rel2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))


def report_phase(path):
    import oracle as O
    from oracle import lda as OL
    z = np.load(path)
    c = CFG
    b = 1 << c["log2b"]
    n, k, Tn = c["n"], c["k"], c["T"]
    rows = []
    T, _, A = synth.planted_symmetric(n, k, c["noise"], c["seed"], dtype=np.float32)
    T64 = T.astype(np.float64)
    ho, go = O.cs_hashes(c["seed"], c["B"], c["log2b"], [n])
    ho, go = ho[:, 0], go[:, 0]
    rows.append(("hash tables h, g (10 x 400)", "entries differing",
                 f"{int(np.sum(z['h'] != ho) + np.sum(z['g'] != go))}", "bit-exact"))
    S64 = np.stack([O.sketch_tensor_sym(T64, ho[m], go[m], b) for m in range(c["B"])])
    Sg = z["S"].astype(np.complex128)
    e_s = max(rel2(Sg[m], S64[m]) for m in range(c["B"]))
    e_smax = max(np.max(np.abs(Sg[m] - S64[m])) / np.max(np.abs(S64[m])) for m in range(c["B"]))
    rows.append(("sketch S (Eq. 7), all 10 sketches", "max rel 2-norm / max-entry",
                 f"{e_s:.2e} / {e_smax:.2e}", "1e-5"))
    # per-sketch contractions, same input sketch (kernel error) and the oracle's own sketch
    U4 = z["U4"].astype(np.float64)
    e_iuu = e_iuu_e2e = e_iuu_ent = 0.0
    e_uuu = e_uuu_e2e = 0.0
    for l in range(U4.shape[0]):
        for m in range(c["B"]):
            got = z["iuu_all"][l, m].astype(np.float64)
            want = O.contract_iuu(Sg[m], U4[l], ho[m], go[m], b, "fft")
            want2 = O.contract_iuu(S64[m], U4[l], ho[m], go[m], b, "fft")
            e_iuu = max(e_iuu, rel2(got, want))
            e_iuu_e2e = max(e_iuu_e2e, rel2(got, want2))
            e_iuu_ent = max(e_iuu_ent, float(np.max(np.abs(got - want)) / np.linalg.norm(want)))
            lw = O.contract_uuu(Sg[m], U4[l], ho[m], go[m], b, "fft")
            lw2 = O.contract_uuu(S64[m], U4[l], ho[m], go[m], b, "fft")
            sc = max(abs(lw), 1e-30)
            e_uuu = max(e_uuu, abs(float(z["uuu_all"][l, m]) - lw) / max(sc, np.linalg.norm(want) * np.linalg.norm(U4[l])))
            e_uuu_e2e = max(e_uuu_e2e, abs(float(z["uuu_all"][l, m]) - lw2) / max(abs(lw2), np.linalg.norm(want2) * np.linalg.norm(U4[l])))
    rows.append(("T^(I,u,u) per sketch (Eq. 14), 4 vectors x 10 sketches",
                 "max rel 2-norm (same sketch / oracle's sketch); max entry / ||v||",
                 f"{e_iuu:.2e} / {e_iuu_e2e:.2e}; {e_iuu_ent:.2e}", "1e-5"))
    rows.append(("T^(u,u,u) per sketch (Eq. 13), 4 x 10", "max |err| / max(|T^|, ||v|| ||u||)",
                 f"{e_uuu:.2e} / {e_uuu_e2e:.2e}", "1e-5"))
    # medians over the sketches (Alg. 1), from the same per-sketch values
    med = np.median(z["iuu_all"].astype(np.float64), axis=1)
    e_med = max(rel2(z["iuu_med"][l], med[l]) for l in range(U4.shape[0]))
    rows.append(("median over sketches of T^(I,u,u)", "max rel 2-norm", f"{e_med:.2e}", "1e-5"))
    # Alg. 1 round by round, chaining the oracle's deflation with the device's (lambda, v)
    S = Sg.copy()
    e_step = e_lam = e_comp = 0.0
    cos_min = 1.0
    U0 = synth.gaussian_inits(k, c["L"], n, c["seed"] + 1).astype(np.float32).astype(np.float64)
    for r in range(k):
        want, _ = O.power_step_sketched(S, z["U_prev_sel"][r].astype(np.float64), ho, go, b, "fft")
        e_step = max(e_step, float(np.linalg.norm(z["U_last_sel"][r] - want)))
        lw, _ = O.eigenvalue_sketched(S, z["V"][r].astype(np.float64), ho, go, b, "fft")
        e_lam = max(e_lam, abs(float(z["lam"][r]) - lw) / max(1.0, abs(lw)))
        # end to end: T oracle power updates of the selected initial vector
        u = U0[r, int(z["tau"][r])]
        u = u / np.linalg.norm(u)
        for _ in range(Tn):
            u, _ = O.power_step_sketched(S, u, ho, go, b, "fft")
        e_comp = max(e_comp, float(np.linalg.norm(z["V"][r] - u)))
        cos_min = min(cos_min, float(abs(np.dot(z["V"][r], u))))
        S = O.deflate_sketches(S, float(z["lam"][r]), z["V"][r].astype(np.float64), ho, go, b, "fft")
    rows.append(("Alg. 1 power update (median + normalise), last step of each round's selected "
                 "vector", "max ||u_gpu - u_oracle(u_gpu prev)||", f"{e_step:.2e}", "1e-4"))
    rows.append(("eigenvalue lambda_r (FP64 median), 20 rounds",
                 "max |err| / max(1, |lambda|)", f"{e_lam:.2e}", "1e-4"))
    rows.append(("component v_r after T = 30 updates from the same start, 20 rounds",
                 "max ||v_gpu - v_oracle||; min |<v_gpu, v_oracle>|", f"{e_comp:.2e}; {cos_min:.6f}",
                 "none (see note)"))
    rows.append(("deflated sketches after 20 rounds (Alg. 1, Eq. 4)", "rel 2-norm",
                 f"{rel2(z['S_deflated'].astype(np.complex128), S):.2e}", "1e-4"))
    # round 0 iterates step by step for three initial vectors
    e_it = 0.0
    Ur = z["U_round0"].astype(np.float64)
    for t in range(Tn):
        for q, tau in enumerate(SAMPLE_TAUS):
            prev = U0[0, tau] / np.linalg.norm(U0[0, tau]) if t == 0 else Ur[t - 1, q]
            want, _ = O.power_step_sketched(Sg, prev, ho, go, b, "fft")
            e_it = max(e_it, float(np.linalg.norm(Ur[t, q] - want)))
    rows.append(("round-0 iterates, every step, 3 vectors", "max ||u_t - oracle(u_{t-1})||",
                 f"{e_it:.2e}", "1e-4"))
    # the synthetic grid cell: Alg. 1 converges, so FP32 and FP64 runs from the same start
    # end at the same components
    e = E1
    b1 = 1 << e["log2b"]
    h1, g1 = O.cs_hashes(e["seed"], e["B"], e["log2b"], [e["n"]])
    h1, g1 = h1[:, 0], g1[:, 0]
    S = z["e1_S"].astype(np.complex128)
    U1 = synth.gaussian_inits(e["k"], e["L"], e["n"], e["seed"] + 3).astype(np.float32).astype(np.float64)
    e_v = e_l = e_lv = 0.0
    moving = []
    for r in range(e["k"]):
        u = U1[r, int(z["e1_tau"][r])]
        u = u / np.linalg.norm(u)
        for _ in range(e["T"]):
            u, _ = O.power_step_sketched(S, u, h1, g1, b1, "fft")
        u_next, _ = O.power_step_sketched(S, u, h1, g1, b1, "fft")
        step = float(np.linalg.norm(u_next - u))
        vg = z["e1_V"][r].astype(np.float64)
        lw, _ = O.eigenvalue_sketched(S, u, h1, g1, b1, "fft")
        lv, _ = O.eigenvalue_sketched(S, vg, h1, g1, b1, "fft")
        e_lv = max(e_lv, abs(float(z["e1_lam"][r]) - lv) / abs(lv))
        if step < 1e-8:      # the oracle's iteration has converged from this start
            e_v = max(e_v, float(np.linalg.norm(vg - u)))
            e_l = max(e_l, abs(float(z["e1_lam"][r]) - lw) / abs(lw))
        else:
            moving.append(f"round {r}: oracle still moving by {step:.1e}, "
                          f"||v_gpu - v_oracle|| = {np.linalg.norm(vg - u):.1e}")
        S = O.deflate_sketches(S, float(z["e1_lam"][r]), vg, h1, g1, b1, "fft")
    conv = e["k"] - len(moving)
    rows.append((f"n = 1000 grid cell (B = 20, b = 2^14): components after T = 30 updates from "
                 f"the same start, the {conv} of 10 rounds whose oracle iteration has converged",
                 "max ||v_gpu - v_oracle||", f"{e_v:.2e}", "—"))
    rows.append(("n = 1000 grid cell: eigenvalues of those rounds, oracle run end to end",
                 "max |err| / |lambda|", f"{e_l:.2e}", "—"))
    rows.append(("n = 1000 grid cell: eigenvalue at the device's component, all 10 rounds",
                 "max |lambda_gpu - lambda_oracle(v_gpu)| / |lambda|", f"{e_lv:.2e}", "1e-4"))
    rows.append(("n = 1000 grid cell: rounds still moving after T = 30 (no fixed point to "
                 "compare)", "oracle's last step; distance", "; ".join(moving) or "none", "—"))
    rows.append(("n = 1000 grid cell: deflated sketches after 10 rounds", "rel 2-norm",
                 f"{rel2(z['e1_S_deflated'].astype(np.complex128), S):.2e}", "1e-4"))
    # spectral LDA
    lc = LDA
    a0 = lc["k"] * lc["alpha"]
    for tag, D in (("full", lc["D_full"]), ("m3", lc["D_m3"])):
        G = z[f"lda_{tag}_gram"]
        rows.append((f"whitening W (V = 50000, k = 100, D = {D})",
                     "max |W^T M2^ W - I| (device M2^ operator)",
                     f"{np.max(np.abs(G - np.eye(lc['k']))):.2e}", "2e-4"))
    cp = synth.lda_corpus(lc["V"], lc["k"], lc["D_m3"], lc["seed"], alpha=lc["alpha"],
                          beta=lc["beta"], mean_len=lc["mean_len"])
    W = z["lda_m3_W"].astype(np.float64)
    M3 = z["lda_m3_M3"].astype(np.float64)
    rng = np.random.default_rng(5)
    e_xxx = e_ixx = 0.0
    for _ in range(4):
        x = rng.standard_normal(lc["k"])
        x /= np.linalg.norm(x)
        xxx, ixx = OL.whitened_m3_contract(cp, W, a0, x)
        g_ixx = np.einsum("abc,b,c->a", M3, x, x)
        g_xxx = float(g_ixx @ x)
        e_ixx = max(e_ixx, rel2(g_ixx, ixx))
        e_xxx = max(e_xxx, abs(g_xxx - xxx) / np.linalg.norm(ixx))
    rows.append((f"M3^(W,W,W) (V = 50000, k = 100, D = {lc['D_m3']}), 4 random unit x",
                 "M3(I,x,x): max rel 2-norm; M3(x,x,x): max |err| / ||M3(I,x,x)||",
                 f"{e_ixx:.2e}; {e_xxx:.2e}", "2e-5 of max entry"))
    print("| result | measure | measured error | test tolerance |")
    print("|---|---|---|---|")
    for row in rows:
        print("| " + " | ".join(row) + " |")


if __name__ == "__main__":
    if len(sys.argv) != 3 or sys.argv[1] not in ("gpu", "report"):
        raise SystemExit(__doc__)
    (gpu_phase if sys.argv[1] == "gpu" else report_phase)(sys.argv[2])
