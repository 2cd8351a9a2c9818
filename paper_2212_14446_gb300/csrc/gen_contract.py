#!/usr/bin/env python3
"""Generate ``contract_gen.cuh``: straight-line device code for the angular parts
of the fast POD descriptors, one specialisation per maximum angular degree PA.

For each PA the generated structs hold
  * ``Mono<PA>::eval``   angular monomials A_x(u) of degree <= PA in the order of
                         the paper's Table 3 (Eq. 23b), each as a product of a
                         lower-degree monomial and one coordinate;
  * ``Mono<PA>::eval2``  the same monomials packed two per float2 (operands of the
                         paired FP32 multiply-add);
  * ``Mono<PA>::grad``   gradient with respect to u of the polynomial
                         sum_x e_x A_x(u)  (used by the adjoint pair pass, Eq. 24c);
  * ``Mono<PA>::dot_grad_deg``  sum_x e_x A_x and its gradient, split by the
                         degree of x (design-matrix columns of D3 and D4_n00);
  * ``Mono<PA>::d3``     three-body contraction sum_l c_nl B_nl^2 per degree n
                         with the multinomial coefficients of Table 4 (Eq. 26a);
  * ``Four<PA>::desc``   four-body descriptors for every partition a >= b >= c
                         with a + b + c <= PA (Table 1 order): b = c = 0 via
                         Eq. 27a, the rest via the trinomial contraction Eq. 30a
                         with equal index triples merged;
  * ``Four<PA>::adjoint`` the derivative of sum_p w_p D4_p (general partitions
                         only) with respect to B.

Everything is emitted as templates on the arithmetic type T so the same code
serves the FP64 and the FP32 paths.  Run:  python gen_contract.py <PAMAX> <out>
"""
import math
import sys
from collections import OrderedDict


def partitions(n):
    """a >= b >= c >= 0 with a + b + c = n, lexicographically descending."""
    out = []
    for a in range(n, -1, -1):
        for b in range(min(a, n - a), -1, -1):
            c = n - a - b
            if 0 <= c <= b:
                out.append((a, b, c))
    return out


def monomials(P):
    """Exponent triples of degree <= P in Table 3 order."""
    res = []
    for n in range(P + 1):
        for lam in partitions(n):
            seen = []
            # assign the parts (largest first) to variables; variables of the
            # first part vary slowest; equal parts take increasing variables
            for v1 in range(3):
                for v2 in range(3):
                    if v2 == v1:
                        continue
                    v3 = 3 - v1 - v2
                    if lam[0] == lam[1] and v1 > v2:
                        continue
                    if lam[1] == lam[2] and v2 > v3:
                        continue
                    e = [0, 0, 0]
                    e[v1], e[v2], e[v3] = lam
                    e = tuple(e)
                    if e not in seen:
                        seen.append(e)
            res.extend(seen)
    return res


def multinomial(e):
    n = sum(e)
    return math.factorial(n) // (math.factorial(e[0]) * math.factorial(e[1]) * math.factorial(e[2]))


def lit(v):
    """Integer-valued constant as a T literal."""
    return f"T({int(v)})"


def gen_pa(PA):
    mons = monomials(PA)
    index = {e: x for x, e in enumerate(mons)}
    NA = len(mons)
    parts = [p for n in range(PA + 1) for p in partitions(n)]
    KA = len(parts)
    L = []
    L.append(f"template <> struct Mono<{PA}> {{")
    L.append(f"  static constexpr int NA = {NA};")
    # --- eval
    L.append("  template <typename T>")
    L.append("  static __device__ __forceinline__ void eval(T ux, T uy, T uz, T* A) {")
    L.append("    A[0] = T(1);")
    names = ["ux", "uy", "uz"]
    for x, e in enumerate(mons):
        if x == 0:
            continue
        d = next(t for t in range(3) if e[t] > 0)
        lower = list(e)
        lower[d] -= 1
        lo = index[tuple(lower)]
        if lo == 0:
            L.append(f"    A[{x}] = {names[d]};")
        else:
            L.append(f"    A[{x}] = A[{lo}] * {names[d]};")
    L.append("  }")
    # --- eval2: the same monomials packed two per float2 (A_x in A2[x / 2].x or .y),
    # the operand layout of the paired FP32 fused multiply-add
    NP2 = (NA + 1) // 2
    L.append(f"  static constexpr int NA2 = {NP2};")
    L.append("  static __device__ __forceinline__ void eval2(float ux, float uy, float uz, float2* A2) {")
    comp = lambda x: f"A2[{x // 2}].{'x' if x % 2 == 0 else 'y'}"
    L.append(f"    {comp(0)} = 1.0f;")
    for x, e in enumerate(mons):
        if x == 0:
            continue
        d = next(t for t in range(3) if e[t] > 0)
        lower = list(e)
        lower[d] -= 1
        lo = index[tuple(lower)]
        if lo == 0:
            L.append(f"    {comp(x)} = {names[d]};")
        else:
            L.append(f"    {comp(x)} = {comp(lo)} * {names[d]};")
    if NA % 2:
        L.append(f"    {comp(NA)} = 0.0f;")
    L.append("  }")
    # --- eval_d: A_x(u) and dA_x = grad A_x . w (forward mode, product rule on the recurrence)
    L.append("  template <typename T>")
    L.append("  static __device__ __forceinline__ void eval_d(T ux, T uy, T uz, T wx, T wy, T wz, T* A, T* dA) {")
    L.append("    A[0] = T(1);")
    L.append("    dA[0] = T(0);")
    wn = ["wx", "wy", "wz"]
    for x, e in enumerate(mons):
        if x == 0:
            continue
        d = next(t for t in range(3) if e[t] > 0)
        lower = list(e)
        lower[d] -= 1
        lo = index[tuple(lower)]
        if lo == 0:
            L.append(f"    A[{x}] = {names[d]};")
            L.append(f"    dA[{x}] = {wn[d]};")
        else:
            L.append(f"    A[{x}] = A[{lo}] * {names[d]};")
            L.append(f"    dA[{x}] = fma(dA[{lo}], {names[d]}, A[{lo}] * {wn[d]});")
    L.append("  }")
    # --- grad of sum_x e_x A_x
    L.append("  template <typename T>")
    L.append("  static __device__ __forceinline__ void grad(const T* e, const T* A, T& gx, T& gy, T& gz) {")
    L.append("    T g0 = T(0), g1 = T(0), g2 = T(0);")
    gn = ["g0", "g1", "g2"]
    for x, ex in enumerate(mons):
        for d in range(3):
            if ex[d] == 0:
                continue
            lower = list(ex)
            lower[d] -= 1
            lo = index[tuple(lower)]
            k = ex[d]
            if k == 1:
                L.append(f"    {gn[d]} = fma(e[{x}], A[{lo}], {gn[d]});")
            else:
                L.append(f"    {gn[d]} = fma({lit(k)} * e[{x}], A[{lo}], {gn[d]});")
    L.append("    gx = g0; gy = g1; gz = g2;")
    L.append("  }")
    # --- degree-resolved dot and gradient: s[n] = sum_{x of degree n} e_x A_x and
    # g[n] = sum_{x of degree n} e_x grad_u A_x (the adjoint rows of the three-body
    # descriptors D3_n are supported on the monomials of degree n)
    L.append("  template <typename T>")
    L.append("  static __device__ __forceinline__ void dot_grad_deg(const T* e, const T* A, T* s, T* gx, T* gy, T* gz) {")
    L.append(f"    for (int n = 0; n <= {PA}; ++n) {{ s[n] = T(0); gx[n] = T(0); gy[n] = T(0); gz[n] = T(0); }}")
    gdn = ["gx", "gy", "gz"]
    for x, ex in enumerate(mons):
        n = sum(ex)
        L.append(f"    s[{n}] = fma(e[{x}], A[{x}], s[{n}]);")
        for d in range(3):
            if ex[d] == 0:
                continue
            lower = list(ex)
            lower[d] -= 1
            lo = index[tuple(lower)]
            k = ex[d]
            if k == 1:
                L.append(f"    {gdn[d]}[{n}] = fma(e[{x}], A[{lo}], {gdn[d]}[{n}]);")
            else:
                L.append(f"    {gdn[d]}[{n}] = fma({lit(k)} * e[{x}], A[{lo}], {gdn[d]}[{n}]);")
    L.append("  }")
    # --- d3 per degree
    L.append("  template <typename T>")
    L.append("  static __device__ __forceinline__ void d3(const T* B, T* d) {")
    for n in range(PA + 1):
        terms = []
        for x, e in enumerate(mons):
            if sum(e) != n:
                continue
            mu = multinomial(e)
            terms.append(f"B[{x}] * B[{x}]" if mu == 1 else f"{lit(mu)} * B[{x}] * B[{x}]")
        L.append(f"    d[{n}] = " + " + ".join(terms) + ";")
    L.append("  }")
    # --- d3 tangent: d3d[n] = 2 sum_{x of degree n} mu_x B_x Bd_x
    L.append("  template <typename T>")
    L.append("  static __device__ __forceinline__ void d3_tangent(const T* B, const T* Bd, T* d) {")
    for n in range(PA + 1):
        terms = []
        for x, e in enumerate(mons):
            if sum(e) != n:
                continue
            terms.append(f"{lit(2 * multinomial(e))} * B[{x}] * Bd[{x}]")
        L.append(f"    d[{n}] = " + " + ".join(terms) + ";")
    L.append("  }")
    # --- d3 adjoint: a_x += 2 h_deg(x) mu_x B_x
    L.append("  template <typename T>")
    L.append("  static __device__ __forceinline__ void d3_adjoint(const T* B, const T* h, T* a) {")
    for x, e in enumerate(mons):
        mu = multinomial(e)
        L.append(f"    a[{x}] = fma({lit(2 * mu)} * h[{sum(e)}], B[{x}], a[{x}]);")
    L.append("  }")
    L.append("};")

    # --- four-body
    L.append(f"template <> struct Four<{PA}> {{")
    L.append(f"  static constexpr int KA = {KA};")
    # index of (n,0,0) partitions
    n00 = [parts.index((n, 0, 0)) for n in range(PA + 1)]
    L.append("  static __device__ __forceinline__ int p_n00(int n) {")
    L.append("    switch (n) {")
    for n in range(PA + 1):
        L.append(f"      case {n}: return {n00[n]};")
    L.append("      default: return -1;")
    L.append("    }")
    L.append("  }")

    def terms_of(a, b, c):
        acc = OrderedDict()
        for q in (e for e in mons if sum(e) == a):
            for s in (e for e in mons if sum(e) == b):
                for t in (e for e in mons if sum(e) == c):
                    x1 = index[tuple(q[i] + s[i] for i in range(3))]
                    x2 = index[tuple(q[i] + t[i] for i in range(3))]
                    x3 = index[tuple(s[i] + t[i] for i in range(3))]
                    key = tuple(sorted((x1, x2, x3)))
                    acc[key] = acc.get(key, 0) + multinomial(q) * multinomial(s) * multinomial(t)
        return acc

    # desc
    L.append("  template <typename T>")
    L.append("  static __device__ __forceinline__ void desc(const T* B, const T* d3, T* D) {")
    nterms = 0
    for p, (a, b, c) in enumerate(parts):
        if b == 0 and c == 0:
            L.append(f"    D[{p}] = B[0] * d3[{a}];")
            continue
        acc = terms_of(a, b, c)
        nterms += len(acc)
        ex = []
        for (x, y, z), k in acc.items():
            t = f"B[{x}] * B[{y}] * B[{z}]"
            ex.append(t if k == 1 else f"{lit(k)} * {t}")
        L.append(f"    D[{p}] = " + " + ".join(ex) + ";")
    L.append("  }")
    # adjoint of sum_p w_p D4_p over the general partitions
    L.append("  template <typename T>")
    L.append("  static __device__ __forceinline__ void adjoint(const T* B, const T* w, T* a) {")
    for p, (a_, b, c) in enumerate(parts):
        if b == 0 and c == 0:
            continue
        acc = terms_of(a_, b, c)
        L.append("    {")
        L.append(f"      const T wp = w[{p}];")
        for (x, y, z), k in acc.items():
            wk = "wp" if k == 1 else f"wk{x}_{y}_{z}"
            if k != 1:
                L.append(f"      const T {wk} = {lit(k)} * wp;")
            L.append(f"      a[{x}] = fma({wk}, B[{y}] * B[{z}], a[{x}]);")
            L.append(f"      a[{y}] = fma({wk}, B[{x}] * B[{z}], a[{y}]);")
            L.append(f"      a[{z}] = fma({wk}, B[{x}] * B[{y}], a[{z}]);")
        L.append("    }")
    L.append("  }")
    # tangent: Dd[p] = sum_x dD4_p/dB_x Bd_x (general partitions by the product rule;
    # b = c = 0 partitions from D4 = B_0 d3_a: Dd = Bd_0 d3_a + B_0 d3d_a)
    L.append("  template <typename T>")
    L.append("  static __device__ __forceinline__ void tangent(const T* B, const T* Bd, const T* d3, const T* d3d, T* Dd) {")
    for p, (a_, b, c) in enumerate(parts):
        if b == 0 and c == 0:
            L.append(f"    Dd[{p}] = fma(Bd[0], d3[{a_}], B[0] * d3d[{a_}]);")
            continue
        acc = terms_of(a_, b, c)
        ex = []
        for (x, y, z), k in acc.items():
            t = f"(Bd[{x}] * B[{y}] * B[{z}] + B[{x}] * Bd[{y}] * B[{z}] + B[{x}] * B[{y}] * Bd[{z}])"
            ex.append(t if k == 1 else f"{lit(k)} * {t}")
        L.append(f"    Dd[{p}] = " + " + ".join(ex) + ";")
    L.append("  }")
    L.append(f"  static constexpr int NTERMS = {nterms};")
    L.append("};")
    return L


def main():
    pamax = int(sys.argv[1]) if len(sys.argv) > 1 else 4
    out = sys.argv[2] if len(sys.argv) > 2 else "contract_gen.cuh"
    lines = ["// Generated by gen_contract.py -- do not edit.",
             "// Angular monomials (Eq. 23b, Table 3), three-body contraction (Eq. 26a, Table 4),",
             "// four-body contraction (Eq. 27a, Eq. 30a) and their adjoints, unrolled per PA.",
             "#pragma once",
             "template <int PA> struct Mono;",
             "template <int PA> struct Four;"]
    for PA in range(pamax + 1):
        lines += gen_pa(PA)
    text = "\n".join(lines) + "\n"
    try:
        with open(out) as f:
            if f.read() == text:
                return
    except FileNotFoundError:
        pass
    with open(out, "w") as f:
        f.write(text)


if __name__ == "__main__":
    main()
