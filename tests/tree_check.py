"""HAPOD-versus-oracle comparison on one tree (host side of the GPU parity tests).

The oracle runs the same recursion (Def. HAPOD) with an exact POD per node
(Householder QR + one-sided Jacobi, FP64) on the very values the GPU consumed.
Checked, with the form's own measured perturbation where floating point can move a
decision:
  * projection error of the root modes <= sum_a eps(a)^2 (Thm. hapod_bound with
    Thm. cor:hapod_bound's local tolerances), times 1.01;
  * every node's rank: the oracle's, or the rank of Def. truncated POD for a
    tolerance whose square lies within m_a ||E_a||_2 of eps(a)^2, E_a the GPU
    form's Gram error on the oracle's input of node a (Weyl: each tail sum moves by
    at most m_a ||E_a||_2);
  * root singular values: |d sigma_j| <= 10 u_eff ||X||_F^2 / sigma_j + 1e-6 sigma_0
    + the size of the modes that entered parents of nodes whose rank differed,
    u_eff = sum_a ||E_a||_2 / ||X||_F^2 (Weyl per node, |d sigma| <= ||E||_2 / (2 sigma));
  * orthonormality of the root modes.
"""
import math

import numpy as np
import torch

import oracle
from tests.helpers import leaf_split, projection_error, rank_within, to_dev, to_host


def hapod_gpu(H, precision, parent, cols, data, n, eps, omega, max_pending=0):
    """Push every leaf (device copies of the same values) in the order of ``data``'s
    keys, return (sigma, U host, stats, status)."""
    dtype = H.DTYPE[precision]
    leaves = list(data)
    ctx = H.hapod_create(parent, cols, eps, omega, n, precision, max_pending_leaves=max_pending)
    bufs = {}
    for a in leaves:
        bufs[a] = to_dev(data[a], dtype=dtype)
        H.hapod_push(ctx, a, bufs[a])
    s, U, st = H.hapod_result(ctx)
    stats = [H.hapod_node_stats(ctx, a) for a in range(len(parent))]
    H.hapod_destroy(ctx)
    return s.numpy(), to_host(U), stats, st


def oracle_tree(parent, cols, data, eps, omega):
    S = sum(cols)
    eps_nodes = oracle.tolerances(parent, cols, eps / math.sqrt(S), omega)
    ref = oracle.hapod(parent, data, eps_nodes, keep_all=True)
    return eps_nodes, ref


def node_input(parent, data, ref, a, f32):
    kids = [b for b in range(len(parent)) if parent[b] == a]
    Xa = data[a] if not kids else np.concatenate([ref[b].Y for b in kids], axis=1)
    if f32:
        Xa = Xa.astype(np.float32).astype(np.float64)
    return np.asfortranarray(Xa)


def check(H, precision, parent, cols, data, X, eps, omega, gpu, oracle_res, ortho_tol, label=""):
    s, Uh, stats, st = gpu
    eps_nodes, ref = oracle_res
    f32 = H.DTYPE[precision] == torch.float32
    root = parent.index(-1)
    fro2 = float(np.sum(X * X))
    bound = sum(e * e for e in eps_nodes)
    perr = projection_error(X, Uh)
    assert perr <= bound * 1.01, (label, perr, bound)
    if ortho_tol is None:  # FP64 forms: U = Y Sigma^-1 loses orthogonality like u (sigma_0 / sigma_k)^2
        ortho_tol = max(1e-12, 1e3 * 2.0 ** -53 * (s[0] / s[-1]) ** 2)
    assert np.max(np.abs(Uh.T @ Uh - np.eye(Uh.shape[1]))) <= ortho_tol, label
    # Gram error of the GPU form on the oracle's input of every node
    e_nodes = []
    for a in range(len(parent)):
        Xa = node_input(parent, data, ref, a, f32)
        if Xa.shape[1] == 0:
            e_nodes.append(0.0)
            continue
        G = H.hapod_gram(to_dev(Xa, dtype=H.DTYPE[precision]), precision).cpu().numpy()
        e_nodes.append(float(np.linalg.norm(G - oracle.gram(Xa), 2)))
    differ = []
    for a in range(len(parent)):
        if stats[a]["k"] == ref[a].N:
            continue
        differ.append(a)
        Xa = node_input(parent, data, ref, a, f32)
        full_s, _, _, _ = oracle.svd(Xa, want_vectors=False)
        assert rank_within(stats[a]["k"], oracle.tail_sums(full_s), eps_nodes[a], Xa.shape[1] * e_nodes[a]), \
            (label, a, stats[a]["k"], ref[a].N)
    u_eff = sum(e_nodes) / fro2
    slack = math.sqrt(sum(eps_nodes[a] ** 2 for a in differ if a != root))
    sr = ref[root].sigma
    k = min(len(s), len(sr))
    dsig = np.abs(s[:k] - sr[:k])
    print(f"{label}: k={len(s)} ref={len(sr)} u_eff={u_eff:.2e} max dsig/s0={dsig.max() / sr[0]:.2e} "
          f"proj={perr / bound:.3f} of bound, nodes with other rank={len(differ)}/{len(parent)}")
    assert abs(len(s) - len(sr)) <= (1 if root in differ else 0), label
    assert np.all(dsig <= 10 * u_eff * fro2 / sr[:k] + 1e-6 * sr[0] + slack), (label, dsig.max(), u_eff)
    return {"u_eff": u_eff, "differ": differ, "proj_frac": perr / bound}


# ------------------------------------------------------------------ full-size waves
def waves_run(H, bench, wl, precision, fro2, stream):
    """bench.run_waves' schedule (device-generated leaves, waves of wl['wave'] leaves,
    max_pending_leaves = wave), returning the root modes too."""
    parent, leaves, cols = bench.c3_tree(wl)
    device = torch.device("cuda", 0)
    gen = bench.Generator(H, wl, H.DTYPE[precision], device, wl["wave"])
    eps = wl["eps_rel"] * math.sqrt(fro2)
    ctx = H.hapod_create(parent, cols, eps, wl["omega"], wl["n"], precision, stream=stream,
                         max_pending_leaves=wl["wave"])
    with torch.cuda.stream(stream):
        for w0 in range(0, len(leaves), wl["wave"]):
            idx = range(w0, min(len(leaves), w0 + wl["wave"]))
            views = {i: gen.gen(i, i - w0, stream) for i in idx}
            for i in idx:
                H.hapod_push(ctx, leaves[i], views[i].t())
        s, U, st = H.hapod_result(ctx, device=device)
    stats = [H.hapod_node_stats(ctx, a) for a in range(len(parent))]
    H.hapod_destroy(ctx)
    del gen
    torch.cuda.synchronize()
    return s.numpy(), U, stats, st


def waves_projection_error(H, bench, wl, U):
    """sum over all snapshots of ||x - Q Q^T x||^2 = ||X||^2 - ||Q^T X||^2 in FP64, Q
    from a QR of the modes, the snapshots regenerated leaf by leaf (FP64 accumulation;
    the cancellation costs about 8 of 16 digits at a relative error of 1e-8)."""
    Q, _ = torch.linalg.qr(U.double())
    gen = bench.Generator(H, wl, torch.float32, U.device, 1)
    cur = torch.cuda.current_stream()
    tot = 0.0
    for i in range(wl["leaves"]):
        X = gen.gen(i, 0, cur).double()  # cols x n
        C = X @ Q                        # cols x k = (Q^T X)^T
        tot += float(torch.sum(X * X) - torch.sum(C * C))
    torch.cuda.synchronize()
    return tot


def full_size_waves(H, bench, wl):
    """Properties that hold at any size, for the fixed-point and the digit-slice FP64
    forms on the full-size device-generated workload: every node's discarded tail
    within its eps(a)^2, the projection error within Thm. hapod_bound's sum of
    eps(a)^2, and the two forms' ranks and root singular values agreeing within the
    fixed-point form's measured Gram error (on a full-size leaf, per unit of trace,
    summed over the nodes) plus the modes of nodes whose ranks differ."""
    stream = torch.cuda.Stream()
    fro2 = bench.c3_fro2(H, wl, torch.device("cuda", 0), stream)
    parent, leaves, cols = bench.c3_tree(wl)
    eps = wl["eps_rel"] * math.sqrt(fro2)
    eps_nodes = oracle.tolerances(parent, cols, eps / math.sqrt(sum(cols)), wl["omega"])
    bound = sum(e * e for e in eps_nodes)
    res = {}
    for form, prec in (("fx3", H.HAPOD_MIXED_FX3), ("fp64_ozaki", H.HAPOD_FP64_OZAKI)):
        s, U, stats, st = waves_run(H, bench, wl, prec, fro2, stream)
        assert st in (H.HAPOD_OK, H.HAPOD_WARN_BELOW_FLOOR), form
        assert all(stats[a]["tail_sq"] <= eps_nodes[a] ** 2 * (1 + 1e-12) for a in range(len(parent))), form
        perr = waves_projection_error(H, bench, wl, U)
        print(f"{wl['name']} {form}: k_root={len(s)} projection error {perr / bound:.4f} of the bound, "
              f"{perr / fro2:.3e} of ||X||^2")
        assert perr <= bound * 1.01, form
        res[form] = (s, stats)
        del U
        torch.cuda.empty_cache()
    gen = bench.Generator(H, wl, torch.float32, torch.device("cuda", 0), 1)
    X = gen.gen(0, 0, torch.cuda.current_stream()).t()
    G1 = H.hapod_gram(X, H.HAPOD_MIXED_FX3)
    G2 = H.hapod_gram(X.double(), H.HAPOD_FP64_OZAKI)
    u_eff = float(torch.linalg.matrix_norm(G1 - G2, ord=2)) / float(torch.trace(G2))
    del gen, X, G1, G2
    (s1, st1), (s2, st2) = res["fx3"], res["fp64_ozaki"]
    differ = [a for a in range(len(parent)) if st1[a]["k"] != st2[a]["k"]]
    print(f"{wl['name']}: u_eff={u_eff:.2e}; nodes with other rank: {len(differ)} of {len(parent)}; "
          f"k_root {len(s1)} / {len(s2)}")
    assert all(abs(st1[a]["k"] - st2[a]["k"]) <= 1 for a in differ)
    assert abs(len(s1) - len(s2)) <= 1
    k = min(len(s1), len(s2))
    slack = math.sqrt(sum(eps_nodes[a] ** 2 for a in differ if parent[a] >= 0))
    dsig = np.abs(s1[:k] - s2[:k])
    assert np.all(dsig <= 10 * u_eff * len(parent) * fro2 / s2[:k] + 1e-6 * s2[0] + slack), dsig.max()
