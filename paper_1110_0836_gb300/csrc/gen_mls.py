"""Generate mls_gen.cuh: straight-line device code for the interpolating cubic MLS fit.

Run `python gen_mls.py` after changing the basis order; the output is committed.

Basis (19 monomials of total degree 1..3 in q = d / lambda_i, Paper II Sec. 2
'third-order polynomial'; the constant term is pinned to U_i by the
interpolating fit).  The kernels order it cubic (0..9), quadratic (10..15),
linear (16..18) so that a Cholesky factorisation M = L L^T followed by back
substitution reaches the linear and quadratic coefficients - the only ones the
derivatives need - first, and never has to compute the cubic ones.

The normal matrix entries are moments  M[a][b] = sum_j w_j q_j^(e_a + e_b),
which take only 80 distinct values (all exponents of total degree 2..6).  Each
moment is accumulated with one fused multiply-add of a weighted monomial w q^beta
(|beta| <= 3) and a monomial q^gamma (1 <= |gamma| <= 3) with beta + gamma = alpha.
"""
from __future__ import annotations

import itertools
import os

CUBIC = [(3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1),
         (0, 1, 2), (0, 0, 3)]
QUAD = [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]
LIN = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
BASIS = CUBIC + QUAD + LIN
NB = len(BASIS)
assert NB == 19
IDX = {e: i for i, e in enumerate(BASIS)}


def add(a, b):
    return tuple(x + y for x, y in zip(a, b))


def sub(a, b):
    return tuple(x - y for x, y in zip(a, b))


def name(e):
    return "xyz"[0] * e[0] + "xyz"[1] * e[1] + "xyz"[2] * e[2]


MOMENTS = sorted({add(a, b) for a in BASIS for b in BASIS}, key=lambda e: (sum(e), [-x for x in e]))
assert len(MOMENTS) == 80
MIDX = {e: i for i, e in enumerate(MOMENTS)}


def split(alpha):
    """(beta index in {-1 (w)} U basis, gamma index in basis) with beta + gamma = alpha.
    Degree >= 4 moments take a cubic beta, so that only w and the ten w q^cubic
    products are needed (degree 4 = cubic + linear, 5 = cubic + quadratic,
    6 = cubic + cubic)."""
    if sum(alpha) <= 3:
        return -1, IDX[alpha]
    for b in BASIS:          # cubic betas come first in the basis order
        if sum(b) != 3:
            continue
        g = sub(alpha, b)
        if min(g) >= 0 and g in IDX:
            return IDX[b], IDX[g]
    raise AssertionError(alpha)


# Packed moment accumulation.  The 80 moments are held as 40 float2
# accumulator pairs.  With the weighted basis pairs wp[k] = w qg2[k] (k < 8),
# degree 2 and 3 are wp[5..7] and wp[0..4] themselves (packed adds).  A packed
# FMA adds two moments of degree 4..6 at once, either as wp[k] * qg2[j]
# ("pair": (w q^(a_k + a_j), w q^(b_k + b_j)) for pairs k = (a_k, b_k),
# j = (a_j, b_j)) or as one half of wp[k] broadcast over qg2[j] ("splat":
# (w q^(h_k + a_j), w q^(h_k + b_j)); a broadcast operand costs no
# instruction).  PRODUCTS lists the ones used for degrees 4, 5 and 6: a
# maximum matching of each degree's moments under such products (7 of 15, 10
# of 21 and 13 of 28 pairs).  The remaining 4 moments take one scalar FMA
# each, two to an accumulator pair: 38 packed and 4 scalar instructions
# instead of 80 scalar ones.
PRODUCTS = [("pair", 0, 8), ("pair", 1, 8), ("pair", 2, 8), ("pair", 6, 6), ("pair", 7, 7),
            ("splat", 3, 1, 8), ("splat", 4, 1, 8),
            ("pair", 0, 5), ("pair", 0, 6), ("pair", 0, 7), ("pair", 1, 6), ("pair", 2, 7),
            ("splat", 3, 1, 5), ("splat", 3, 1, 7), ("splat", 4, 1, 5), ("splat", 4, 1, 7),
            ("splat", 6, 1, 3),
            ("pair", 0, 0), ("pair", 0, 1), ("pair", 0, 2), ("pair", 1, 1), ("pair", 2, 2),
            ("pair", 4, 4), ("splat", 1, 1, 3), ("splat", 1, 1, 4), ("splat", 2, 1, 4),
            ("splat", 3, 0, 3), ("splat", 3, 0, 4), ("splat", 3, 1, 0), ("splat", 4, 1, 0)]
NWP = 8  # weighted pairs formed (w q for basis pairs 0..7: cubic and quadratic)


def packed_moment_layout():
    """[(kind, operands, (alpha_x, alpha_y))] per accumulator pair, and alpha -> (pair, half)."""
    bp = [(BASIS[2 * j], BASIS[2 * j + 1] if 2 * j + 1 < NB else None) for j in range(10)]
    pairs = [("add", k, bp[k]) for k in (5, 6, 7, 0, 1, 2, 3, 4)]
    for prod in PRODUCTS:
        if prod[0] == "pair":
            _, k, j = prod
            h = (add(bp[k][0], bp[j][0]), add(bp[k][1], bp[j][1]))
        else:
            _, k, hk, j = prod
            h = (add(bp[k][hk], bp[j][0]), add(bp[k][hk], bp[j][1]))
        assert h[0] != h[1] and sum(h[0]) == sum(h[1]) >= 4
        pairs.append((prod[0], prod[1:], h))
    done = [a for p in pairs for a in p[2]]
    assert len(done) == len(set(done)) == 76
    singles = [a for a in MOMENTS if a not in set(done)]
    assert len(singles) == 4
    for i in range(0, 4, 2):
        pairs.append(("single", None, (singles[i], singles[i + 1])))
    assert len(pairs) == 40
    pos = {}
    for p, (_, _, h) in enumerate(pairs):
        for half, a in enumerate(h):
            pos[a] = (p, "xy"[half])
    assert sorted(pos) == sorted(MOMENTS)
    return pairs, pos


def gen_packed_moments(w):
    pairs, pos = packed_moment_layout()
    w("constexpr int kNM2 = 40;  // float2 accumulator pairs of the 80 moments (packed layout)")
    w("constexpr int kNWP = 8;   // weighted basis pairs w qg2[k], k < 8")
    w("")
    w("// wp[k] = w qg2[k] for the cubic and quadratic basis pairs.")
    w("__device__ __forceinline__ void mls_weight_pairs(const float2 (&qg2)[kNB2], float wt, float2 (&wp)[kNWP]) {")
    w("  const float2 w2 = make_float2(wt, wt);")
    w("#pragma unroll")
    w("  for (int k = 0; k < kNWP; ++k) wp[k] = __fmul2_rn(qg2[k], w2);")
    w("}")
    w("")
    w("// m2 += w q^alpha for the 80 moments in the packed layout: 8 packed adds,")
    w("// 30 packed FMAs (a broadcast half of wp in 13 of them) and 4 scalar FMAs.")
    w("__device__ __forceinline__ void mls_accum_moments_p2(const float2 (&qg2)[kNB2], const float2 (&wp)[kNWP], float2 (&m2)[kNM2]) {")
    for p, (kind, op, h) in enumerate(pairs):
        if kind == "add":
            w(f"  m2[{p}] = __fadd2_rn(m2[{p}], wp[{op}]);  // {name(h[0])}, {name(h[1])}")
        elif kind == "pair":
            w(f"  m2[{p}] = __ffma2_rn(wp[{op[0]}], qg2[{op[1]}], m2[{p}]);  // {name(h[0])}, {name(h[1])}")
        elif kind == "splat":
            k, hk, j = op
            c = f"wp[{k}].{'xy'[hk]}"
            w(f"  m2[{p}] = __ffma2_rn(make_float2({c}, {c}), qg2[{j}], m2[{p}]);  // {name(h[0])}, {name(h[1])}")
        else:
            for half, a in zip("xy", h):
                b, g = split(a)
                assert b >= 0 and b < 2 * NWP
                w(f"  m2[{p}].{half} = fmaf(wp[{b // 2}].{'xy'[b % 2]}, qg2[{g // 2}].{'xy'[g % 2]}, m2[{p}].{half});  // {name(a)}")
    w("}")
    w("")
    w("// Normal matrix, packed lower triangle, from the packed moment layout.")
    w("template <typename MT>")
    w("__device__ __forceinline__ void mls_assemble_p2(const float2 (&m2)[kNM2], MT& M) {")
    for r in range(NB):
        for c in range(r + 1):
            p, half = pos[add(BASIS[r], BASIS[c])]
            w(f"  M[{tri(r, c)}] = m2[{p}].{half};")
    w("}")
    w("")


def tri(r, c):
    """packed lower-triangle index of (r, c), r >= c"""
    return r * (r + 1) // 2 + c


def gen():
    L = []
    w = L.append
    w("// Generated by gen_mls.py - do not edit.  Straight-line pieces of the")
    w("// interpolating cubic MLS fit (basis order cubic, quadratic, linear).")
    w("#pragma once")
    w("namespace phb {")
    w(f"constexpr int kNB = {NB};      // basis size")
    w(f"constexpr int kNM = {len(MOMENTS)};      // distinct moments (degree 2..6)")
    w(f"constexpr int kNT = {NB * (NB + 1) // 2};     // packed lower triangle")
    w("constexpr int kLin0 = 16;   // first linear basis index (x, y, z)")
    w("constexpr int kQuad0 = 10;  // first quadratic index (xx, xy, xz, yy, yz, zz)")
    w("")
    # monomials
    w("// q^gamma for the 19 basis monomials, and w q^beta for beta in {0} U basis.")
    w("template <typename T>")
    w("__device__ __forceinline__ void mls_monomials(T x, T y, T z, T wt, T (&qg)[kNB], T (&wq)[kNB + 1]) {")
    w("  const T xx = x * x, xy = x * y, xz = x * z, yy = y * y, yz = y * z, zz = z * z;")
    vals = {(1, 0, 0): "x", (0, 1, 0): "y", (0, 0, 1): "z", (2, 0, 0): "xx", (1, 1, 0): "xy",
            (1, 0, 1): "xz", (0, 2, 0): "yy", (0, 1, 1): "yz", (0, 0, 2): "zz"}
    cubic_expr = {(3, 0, 0): "xx * x", (2, 1, 0): "xx * y", (2, 0, 1): "xx * z", (1, 2, 0): "xy * y",
                  (1, 1, 1): "xy * z", (1, 0, 2): "xz * z", (0, 3, 0): "yy * y", (0, 2, 1): "yy * z",
                  (0, 1, 2): "yz * z", (0, 0, 3): "zz * z"}
    for i, e in enumerate(BASIS):
        expr = cubic_expr.get(e, vals.get(e))
        w(f"  qg[{i}] = {expr};  // {name(e)}")
    w("  wq[0] = wt;")
    for i in range(NB):
        w(f"  wq[{i + 1}] = wt * qg[{i}];")
    w("}")
    w("")
    w("// q^gamma for the 19 basis monomials, w, and w q^beta for the ten cubic")
    w("// betas only (all that mls_accum_moments reads); wq[11..19] are not set.")
    w("template <typename T>")
    w("__device__ __forceinline__ void mls_monomials_cubic_w(T x, T y, T z, T wt, T (&qg)[kNB], T (&wq)[kNB + 1]) {")
    w("  const T xx = x * x, xy = x * y, xz = x * z, yy = y * y, yz = y * z, zz = z * z;")
    for i, e in enumerate(BASIS):
        expr = cubic_expr.get(e, vals.get(e))
        w(f"  qg[{i}] = {expr};  // {name(e)}")
    w("  wq[0] = wt;")
    for i, e in enumerate(BASIS):
        if sum(e) == 3:
            w(f"  wq[{i + 1}] = wt * qg[{i}];")
    w("}")
    w("")
    w("// q^gamma for the 19 basis monomials only.")
    w("template <typename T>")
    w("__device__ __forceinline__ void mls_basis(T x, T y, T z, T (&qg)[kNB]) {")
    w("  const T xx = x * x, xy = x * y, xz = x * z, yy = y * y, yz = y * z, zz = z * z;")
    for i, e in enumerate(BASIS):
        expr = cubic_expr.get(e, vals.get(e))
        w(f"  qg[{i}] = {expr};  // {name(e)}")
    w("}")
    w("")
    # ---- FP32 paired forms: the basis as ten float2 pairs (q^gamma of basis
    # indices 2j, 2j+1; the last pair holds q^gamma_18 and 0), so that the
    # right-hand-side sums take packed FP32x2 fused multiply-adds
    w("constexpr int kNB2 = (kNB + 1) / 2;  // float2 pairs of the basis")
    w("")
    w("// The 19 basis monomials as float2 pairs (qg2[9].y = 0).")
    w("__device__ __forceinline__ void mls_basis2(float x, float y, float z, float2 (&qg2)[kNB2]) {")
    w("  const float xx = x * x, xy = x * y, xz = x * z, yy = y * y, yz = y * z, zz = z * z;")
    exprs = [cubic_expr.get(e, vals.get(e)) for e in BASIS] + ["0.f"]
    for j in range(10):
        w(f"  qg2[{j}] = make_float2({exprs[2 * j]}, {exprs[2 * j + 1]});")
    w("}")
    w("")
    w("// b2 += q^beta (w du) for the basis pairs: ten packed FP32x2 FMAs (the")
    w("// second half of b2[9] accumulates 0).")
    w("__device__ __forceinline__ void mls_accum_rhs_basis2(const float2 (&qg2)[kNB2], float wdu, float2 (&b2)[kNB2]) {")
    w("  const float2 s = make_float2(wdu, wdu);")
    w("#pragma unroll")
    w("  for (int j = 0; j < kNB2; ++j) b2[j] = __ffma2_rn(qg2[j], s, b2[j]);")
    w("}")
    w("")
    w("// p(q).c for the paired basis and coefficients (two partial sums).")
    w("__device__ __forceinline__ float mls_dot2(const float2 (&qg2)[kNB2], const float2 (&c2)[kNB2]) {")
    w("  float2 acc = make_float2(0.f, 0.f);")
    w("#pragma unroll")
    w("  for (int j = 0; j < kNB2; ++j) acc = __ffma2_rn(qg2[j], c2[j], acc);")
    w("  return acc.x + acc.y;")
    w("}")
    w("")
    gen_packed_moments(w)
    w("// m[alpha] += w q^alpha for the 80 moments.")
    w("template <typename T>")
    w("__device__ __forceinline__ void mls_accum_moments(const T (&qg)[kNB], const T (&wq)[kNB + 1], T (&m)[kNM]) {")
    for a, alpha in enumerate(MOMENTS):
        b, g = split(alpha)
        w(f"  m[{a}] = fma(wq[{b + 1}], qg[{g}], m[{a}]);  // {name(alpha)}")
    w("}")
    w("")
    w("// b[beta] += w q^beta du for the 19 basis monomials.")
    w("template <typename T>")
    w("__device__ __forceinline__ void mls_accum_rhs(const T (&wq)[kNB + 1], T du, T (&b)[kNB]) {")
    for i in range(NB):
        w(f"  b[{i}] = fma(wq[{i + 1}], du, b[{i}]);")
    w("}")
    w("")
    w("// b[beta] += q^beta (w du) for the 19 basis monomials (weight folded into du).")
    w("template <typename T>")
    w("__device__ __forceinline__ void mls_accum_rhs_basis(const T (&qg)[kNB], T wdu, T (&b)[kNB]) {")
    for i in range(NB):
        w(f"  b[{i}] = fma(qg[{i}], wdu, b[{i}]);")
    w("}")
    w("")
    w("// Normal matrix, packed lower triangle: M[tri(r,c)] = m[e_r + e_c].")
    w("template <typename MMT, typename MT>")
    w("__device__ __forceinline__ void mls_assemble(const MMT& m, MT& M) {")
    for r in range(NB):
        for c in range(r + 1):
            w(f"  M[{tri(r, c)}] = m[{MIDX[add(BASIS[r], BASIS[c])]}];")
    w("}")
    w("")
    w("// For each moment alpha one basis pair (r, c), r >= c, with e_r + e_c = alpha")
    w("// (to read the moments out of a full Gram matrix of the basis).")
    w("__device__ __forceinline__ void mls_moment_pair(int a, int& r, int& c) {")
    reps = []
    for alpha in MOMENTS:
        found = None
        for r in range(NB):
            for c in range(r + 1):
                if add(BASIS[r], BASIS[c]) == alpha:
                    found = (r, c)
                    break
            if found:
                break
        reps.append(found)
    w("  constexpr unsigned char t[kNM][2] = {")
    for k in range(0, len(reps), 10):
        w("    " + ", ".join(f"{{{r}, {c}}}" for r, c in reps[k:k + 10]) + ",")
    w("  };")
    w("  r = t[a][0];")
    w("  c = t[a][1];")
    w("}")
    w("")
    w("// Index of moment e_r + e_c (for kernels that read moments from memory).")
    w("__device__ __forceinline__ int mls_moment_index(int r, int c) {")
    w("  constexpr unsigned char t[kNT] = {")
    row = []
    for r in range(NB):
        for c in range(r + 1):
            row.append(str(MIDX[add(BASIS[r], BASIS[c])]))
    for k in range(0, len(row), 20):
        w("    " + ", ".join(row[k:k + 20]) + ",")
    w("  };")
    w("  return r >= c ? t[r * (r + 1) / 2 + c] : t[c * (c + 1) / 2 + r];")
    w("}")
    w("")
    # Cholesky
    w("// In-place Cholesky of the packed normal matrix.  On return the packed")
    w("// array holds L (strict lower part; the diagonal entries keep M_kk) and")
    w("// inv_diag[k] = 1 / L_kk.  Returns the smallest pivot L_kk^2 seen (<= 0:")
    w("// not positive definite).  MT / DT: arrays or array-like accessors.")
    w("template <typename T, typename MT, typename DT>")
    w("__device__ __forceinline__ T mls_cholesky(MT& M, DT& inv_diag) {")
    w("  T minpiv = M[0];")
    for j in range(NB):
        terms = "".join(f" - M[{tri(j, k)}] * M[{tri(j, k)}]" for k in range(j))
        if j == 0:
            w(f"  {{ T s = M[{tri(0, 0)}];")
        else:
            w(f"  {{ T s = M[{tri(j, j)}];")
            for k in range(j):
                w(f"    s = fma(-M[{tri(j, k)}], M[{tri(j, k)}], s);")
        w("    minpiv = s < minpiv ? s : minpiv;")
        w(f"    const T r = phb_rsqrt(s > T(0) ? s : T(1));")
        w(f"    inv_diag[{j}] = r;")
        for i in range(j + 1, NB):
            w(f"    {{ T v = M[{tri(i, j)}];")
            for k in range(j):
                w(f"      v = fma(-M[{tri(i, k)}], M[{tri(j, k)}], v);")
            w(f"      M[{tri(i, j)}] = v * r; }}")
        w("  }")
    w("  return minpiv;")
    w("}")
    w("")
    w("// Estimate of ||M_s^-1||_inf for the Jacobi-scaled normal matrix")
    w("// M_s = D M D, D = diag(M_kk^-1/2), from the factor of M as left by")
    w("// mls_cholesky: one forward substitution L y = D^-1 b whose right-hand side")
    w("// signs b_k = +-1 are chosen, row by row, to make |y_k| grow (the greedy")
    w("// choice of the LINPACK condition estimator), one back substitution")
    w("// L^T x = y, and max_k |x_k| sqrt(M_kk) = ||M_s^-1 b||_inf.  A lower bound of")
    w("// the norm that tracks it closely for the normal matrices of the fit.")
    w("template <typename T, typename MT, typename DT>")
    w("__device__ __forceinline__ T mls_inv_norm_est(const MT& M, const DT& inv_diag) {")
    w(f"  T y[{NB}], sq[{NB}];")
    for i in range(NB):
        w(f"  sq[{i}] = sqrt(M[{tri(i, i)}]);")
    for i in range(NB):
        w(f"  {{ T s = T(0);")
        for k in range(i):
            w(f"    s = fma(M[{tri(i, k)}], y[{k}], s);")
        w(f"    y[{i}] = ((s > T(0) ? -sq[{i}] : sq[{i}]) - s) * inv_diag[{i}]; }}")
    for i in reversed(range(NB)):
        w(f"  {{ T v = y[{i}];")
        for k in range(i + 1, NB):
            w(f"    v = fma(-M[{tri(k, i)}], y[{k}], v);")
        w(f"    y[{i}] = v * inv_diag[{i}]; }}")
    w("  T mx = T(0);")
    for i in range(NB):
        w(f"  mx = fmax(mx, fabs(y[{i}]) * sq[{i}]);")
    w("  return mx;")
    w("}")
    w("")
    w("// Forward substitution L y = b in place (b becomes y).")
    w("template <typename MT, typename DT, typename BT>")
    w("__device__ __forceinline__ void mls_forward(const MT& L, const DT& inv_diag, BT& b) {")
    for i in range(NB):
        w(f"  {{ auto v = b[{i}];")
        for k in range(i):
            w(f"    v = fma(-L[{tri(i, k)}], b[{k}], v);")
        w(f"    b[{i}] = v * inv_diag[{i}]; }}")
    w("}")
    w("")
    w("// Back substitution L^T c = y for the last 9 unknowns only (quadratic and")
    w("// linear coefficients); y[10..18] becomes c[10..18].")
    w("template <typename MT, typename DT, typename BT>")
    w("__device__ __forceinline__ void mls_back9(const MT& L, const DT& inv_diag, BT& y) {")
    for i in range(NB - 1, 9, -1):
        w(f"  {{ auto v = y[{i}];")
        for k in range(i + 1, NB):
            w(f"    v = fma(-L[{tri(k, i)}], y[{k}], v);")
        w(f"    y[{i}] = v * inv_diag[{i}]; }}")
    w("}")
    w("")
    w("// Full back substitution L^T c = y (all 19 coefficients).")
    w("template <typename MT, typename DT, typename BT>")
    w("__device__ __forceinline__ void mls_back19(const MT& L, const DT& inv_diag, BT& y) {")
    for i in range(NB - 1, -1, -1):
        w(f"  {{ auto v = y[{i}];")
        for k in range(i + 1, NB):
            w(f"    v = fma(-L[{tri(k, i)}], y[{k}], v);")
        w(f"    y[{i}] = v * inv_diag[{i}]; }}")
    w("}")
    w("")
    # ---- the same triangular solves for two right-hand sides at once (FP32
    # pairs: b2[i] = (first field's b[i], second field's b[i])), packed FMAs
    # with the factor's entries broadcast; each half rounds exactly as the
    # scalar form
    w("// mls_forward for two right-hand sides in the halves of b2.")
    w("template <typename MT, typename DT>")
    w("__device__ __forceinline__ void mls_forward2(const MT& L, const DT& inv_diag, float2 (&b)[kNB]) {")
    for i in range(NB):
        w(f"  {{ float2 v = b[{i}];")
        for k in range(i):
            w(f"    v = __ffma2_rn(make_float2(-L[{tri(i, k)}], -L[{tri(i, k)}]), b[{k}], v);")
        w(f"    b[{i}] = __fmul2_rn(v, make_float2(inv_diag[{i}], inv_diag[{i}])); }}")
    w("}")
    w("")
    for nm_, lo in (("mls_back9_2", 10), ("mls_back19_2", 0)):
        w(f"// {nm_[:-2]} for two right-hand sides in the halves of y2.")
        w("template <typename MT, typename DT>")
        w(f"__device__ __forceinline__ void {nm_}(const MT& L, const DT& inv_diag, float2 (&y)[kNB]) {{")
        for i in range(NB - 1, lo - 1, -1):
            w(f"  {{ float2 v = y[{i}];")
            for k in range(i + 1, NB):
                w(f"    v = __ffma2_rn(make_float2(-L[{tri(k, i)}], -L[{tri(k, i)}]), y[{k}], v);")
            w(f"    y[{i}] = __fmul2_rn(v, make_float2(inv_diag[{i}], inv_diag[{i}])); }}")
        w("}")
        w("")
    # ---- adjoint helpers: all monomials of degree 0..6 and polynomial gradients
    MONO = sorted({(a, b, c) for a in range(7) for b in range(7) for c in range(7) if a + b + c <= 6},
                  key=lambda e: (sum(e), [-x for x in e]))
    assert len(MONO) == 84
    MO = {e: i for i, e in enumerate(MONO)}
    w("constexpr int kNMono = 84;  // monomials of total degree 0..6")
    w("")
    w("// All monomials q^a of total degree 0..6 (graded order, mono[0] = 1).")
    w("template <typename T>")
    w("__device__ __forceinline__ void mls_monos6(T x, T y, T z, T (&mono)[kNMono]) {")
    w("  mono[0] = T(1);")
    for e in MONO[1:]:
        # build from a lower monomial times one coordinate
        for ax, nm in ((0, "x"), (1, "y"), (2, "z")):
            if e[ax] > 0:
                lower = list(e); lower[ax] -= 1
                w(f"  mono[{MO[e]}] = mono[{MO[tuple(lower)]}] * {nm};  // {name(e)}")
                break
    w("}")
    w("")
    w("// P = sum_alpha mbar[alpha] q^alpha over the 80 moments and its gradient in q.")
    w("template <typename T, typename MB>")
    w("__device__ __forceinline__ void mls_eval_moment_poly(const T (&mono)[kNMono], const MB& mbar, T& P, T& Px, T& Py, T& Pz) {")
    w("  T p = T(0), px = T(0), py = T(0), pz = T(0);")
    for a, al in enumerate(MOMENTS):
        w(f"  {{ const T c = mbar[{a}];")
        w(f"    p = fma(c, mono[{MO[al]}], p);")
        for ax, acc in ((0, "px"), (1, "py"), (2, "pz")):
            if al[ax] > 0:
                lo = list(al); lo[ax] -= 1
                coef = f"T({al[ax]}) * " if al[ax] > 1 else ""
                w(f"    {acc} = fma({coef}c, mono[{MO[tuple(lo)]}], {acc});")
        w("  }")
    w("  P = p; Px = px; Py = py; Pz = pz;")
    w("}")
    w("")
    w("// V = sum_beta B[beta] p_beta(q) over the 19 basis monomials and its gradient in q.")
    w("template <typename T, typename BB>")
    w("__device__ __forceinline__ void mls_eval_basis_poly(const T (&mono)[kNMono], const BB& B, T& V, T& Vx, T& Vy, T& Vz) {")
    w("  T v = T(0), vx = T(0), vy = T(0), vz = T(0);")
    for i, be in enumerate(BASIS):
        w(f"  {{ const T c = B[{i}];")
        w(f"    v = fma(c, mono[{MO[be]}], v);")
        for ax, acc in ((0, "vx"), (1, "vy"), (2, "vz")):
            if be[ax] > 0:
                lo = list(be); lo[ax] -= 1
                coef = f"T({be[ax]}) * " if be[ax] > 1 else ""
                w(f"    {acc} = fma({coef}c, mono[{MO[tuple(lo)]}], {acc});")
        w("  }")
    w("  V = v; Vx = vx; Vy = vy; Vz = vz;")
    w("}")
    w("")
    w("// Adjoint of the normal matrix through its moments:")
    w("// mbar[e_r + e_c] -= bbar[r] * c[c] for all r, c (one right-hand side).")
    w("template <typename T, typename BT, typename CT>")
    w("__device__ __forceinline__ void mls_accum_mbar(const BT& bbar, const CT& c, T (&mbar)[kNM]) {")
    for r in range(NB):
        for cc in range(NB):
            w(f"  mbar[{MIDX[add(BASIS[r], BASIS[cc])]}] = fma(-bbar[{r}], c[{cc}], mbar[{MIDX[add(BASIS[r], BASIS[cc])]}]);")
    w("}")
    w("")
    w("// The 19 basis values from the monomial table.")
    w("template <typename T>")
    w("__device__ __forceinline__ void mls_basis_from_monos(const T (&mono)[kNMono], T (&p)[kNB]) {")
    for i, be in enumerate(BASIS):
        w(f"  p[{i}] = mono[{MO[be]}];")
    w("}")
    w("")
    w("// Basis value p_beta(q) from the monomial table.")
    w("__device__ __forceinline__ int mls_basis_mono(int i) {")
    w("  constexpr unsigned char t[kNB] = {" + ", ".join(str(MO[b]) for b in BASIS) + "};")
    w("  return t[i];")
    w("}")
    w("}  // namespace phb")
    return "\n".join(L) + "\n"


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mls_gen.cuh")
    with open(out, "w") as f:
        f.write(gen())
    print(out)
