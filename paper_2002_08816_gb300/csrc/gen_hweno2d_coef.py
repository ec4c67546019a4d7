"""Generates hweno2d_coef.cuh: the 2D reconstruction of Zhao & Qiu,
arXiv:2002.08816, Sec. 2.2 Step 5, as straight-line device code.

Run once (needs sympy); the outputs are committed:

    python gen_hweno2d_coef.py > hweno2d_coef.cuh
    python gen_hweno2d_coef.py adjoint > hweno2d_adj_coef.cuh

The second file holds what the adjoint kernels need: the transposes of the
point maps (g[j] += sum_p M[p][j] l[p]) and the gradients of the smoothness
indicators (g += s grad beta(d), from the same LDL^T forms).

Everything is derived in exact arithmetic from the moment conditions the paper
states, in the reference coordinates xi = (x - x_i)/dx, eta = (y - y_j)/dy:
  p0: quartic matching the nine cell averages and the centre's first moments
      exactly, the first moments of cells 2, 4, 6, 8 in least squares (KKT);
  p1..p4: quadratics on the 2x2 stencils {1,2,4,5}, {2,3,5,6}, {4,5,7,8},
      {5,6,8,9} matching four averages and the centre's first moments;
  beta_n: Eq. (2dGHYZ) for square cells (dx = dy), written as a sum of
      weighted squares of linear forms in the data (an exact LDL^T of the
      Gram matrix of the derivatives).
Data order: ubar of cells 1..9, vbar of cells 2,4,5,6,8, wbar of cells
2,4,5,6,8 (cells numbered as in the paper's Fig. 1).  Point order per cell:
left face (xi = -1/2) at eta_k, right face, bottom face (eta = -1/2) at xi_k,
top face, then the interior (xi_k, eta_l) with k fastest.
"""

import sys

import sympy as sp

xi, eta = sp.symbols("xi eta")
CELLS = {1: (-1, -1), 2: (0, -1), 3: (1, -1), 4: (-1, 0), 5: (0, 0), 6: (1, 0),
         7: (-1, 1), 8: (0, 1), 9: (1, 1)}
MOM = [2, 4, 5, 6, 8]
HALF = sp.Rational(1, 2)


def monomials(deg):
    return [xi ** a * eta ** (d - a) for d in range(deg + 1) for a in range(d, -1, -1)]


def moment(expr, kind, cell):
    di, dj = CELLS[cell]
    w = 1 if kind == "avg" else ((xi - di) if kind == "xm" else (eta - dj))
    return sp.integrate(sp.integrate(expr * w, (xi, di - HALF, di + HALF)),
                        (eta, dj - HALF, dj + HALF))


def data_index(kind, cell):
    if kind == "avg":
        return cell - 1
    return 9 + (0 if kind == "xm" else 5) + MOM.index(cell)


def p0_map():
    """15 x 19 rational matrix: quartic coefficients from the data."""
    mons = monomials(4)
    eq = [("avg", c) for c in range(1, 10)] + [("xm", 5), ("ym", 5)]
    ls = [("xm", c) for c in (2, 4, 6, 8)] + [("ym", c) for c in (2, 4, 6, 8)]
    E = sp.Matrix([[moment(m, k, c) for m in mons] for k, c in eq])
    A = sp.Matrix([[moment(m, k, c) for m in mons] for k, c in ls])
    K = sp.zeros(26, 26)
    K[:15, :15] = A.T * A
    K[:15, 15:] = E.T
    K[15:, :15] = E
    Ki = K.inv()
    M = sp.zeros(15, 19)
    AT = Ki[:15, :15] * A.T
    for r, (k, c) in enumerate(ls):
        for p in range(15):
            M[p, data_index(k, c)] += AT[p, r]
    for r, (k, c) in enumerate(eq):
        for p in range(15):
            M[p, data_index(k, c)] += Ki[p, 15 + r]
    return M


STENCILS = {1: (1, 2, 4, 5), 2: (2, 3, 5, 6), 3: (4, 5, 7, 8), 4: (5, 6, 8, 9)}


def quad_map(n):
    mons = monomials(2)
    conds = [("avg", c) for c in STENCILS[n]] + [("xm", 5), ("ym", 5)]
    Q = sp.Matrix([[moment(m, k, c) for m in mons] for k, c in conds])
    Qi = Q.inv()
    M = sp.zeros(6, 19)
    for r, (k, c) in enumerate(conds):
        for p in range(6):
            M[p, data_index(k, c)] += Qi[p, r]
    return M


def gram(deg):
    """Eq. (2dGHYZ) for dx = dy: beta = c^T B c over the monomials of degree <= deg."""
    mons = monomials(deg)
    n = len(mons)
    B = sp.zeros(n, n)
    for l1 in range(deg + 1):
        for l2 in range(deg + 1 - l1):
            if l1 + l2 == 0:
                continue
            ders = [sp.diff(m, xi, l1, eta, l2) if (l1 or l2) else m for m in mons]
            for p in range(n):
                for q in range(p, n):
                    v = sp.integrate(sp.integrate(ders[p] * ders[q], (xi, -HALF, HALF)),
                                     (eta, -HALF, HALF))
                    B[p, q] += v
                    if q != p:
                        B[q, p] += v
    return B


def ldl_forms(B, M):
    """beta = d^T (M^T B M) d as sum_k D_k (l_k . d)^2 via an exact LDL^T of B
    without its first row and column (the constant monomial has no derivative)."""
    Bs = B[1:, 1:]
    n = Bs.shape[0]
    L = sp.eye(n)
    D = [0] * n
    for j in range(n):
        D[j] = Bs[j, j] - sum(L[j, k] ** 2 * D[k] for k in range(j))
        for i in range(j + 1, n):
            L[i, j] = (Bs[i, j] - sum(L[i, k] * L[j, k] * D[k] for k in range(j))) / D[j]
    Ms = M[1:, :]
    forms = (L.T * Ms)
    return [sp.nsimplify(d) for d in D], forms


def points(ng):
    if ng == 3:
        g = [-sp.sqrt(15) / 10, sp.Integer(0), sp.sqrt(15) / 10]
    else:
        g = [-sp.sqrt(3) / 6, sp.sqrt(3) / 6]
    pts = [(-HALF, e) for e in g] + [(HALF, e) for e in g] + [(x, -HALF) for x in g] + \
          [(x, HALF) for x in g] + [(gk, gl) for gl in g for gk in g]
    return pts


def value_map(M, deg, pts):
    mons = monomials(deg)
    rows = []
    for (x, y) in pts:
        vals = [m.subs({xi: x, eta: y}) for m in mons]
        rows.append([sp.nsimplify(sp.expand(sum(vals[k] * M[k, j] for k in range(len(mons)))))
                     for j in range(19)])
    return rows


def lit(v):
    f = sp.N(v, 25)
    if f == 0:
        return None
    return "R(%s)" % sp.Float(f, 20)


def emit_map(name, rows, nd_in="d", out="o"):
    lines = ["template <typename R>",
             "__device__ __forceinline__ void %s(const R* %s, R* %s) {" % (name, nd_in, out)]
    for p, row in enumerate(rows):
        terms = []
        for j, v in enumerate(row):
            s = lit(v)
            if s is not None:
                terms.append("%s * %s[%d]" % (s, nd_in, j))
        lines.append("  %s[%d] = %s;" % (out, p, " + ".join(terms) if terms else "R(0)"))
    lines.append("}")
    return "\n".join(lines)


def emit_map_x2(name, rows):
    """The same map on pairs of FP32 data (two components of one cell), in
    packed FP32 arithmetic: each coefficient is a broadcast pair and every
    term one packed fma, so a pair of values costs the instructions of one;
    the terms run in the order of emit_map's, the first a product."""
    lines = ["__device__ __forceinline__ void %s(const float2* d, float2* o) {" % name,
             "  float2 a;"]
    for p, row in enumerate(rows):
        first = True
        for j, v in enumerate(row):
            s = lit(v)
            if s is None:
                continue
            c = "hw2_pair(%s)" % s[2:-1]
            if first:
                lines.append("  a = __fmul2_rn(%s, d[%d]);" % (c, j))
                first = False
            else:
                lines.append("  a = __ffma2_rn(%s, d[%d], a);" % (c, j))
        if first:
            lines.append("  a = make_float2(0.0f, 0.0f);")
        lines.append("  o[%d] = a;" % p)
    lines.append("}")
    return "\n".join(lines)


def emit_beta(name, D, forms):
    lines = ["template <typename R>",
             "__device__ __forceinline__ R %s(const R* d) {" % name,
             "  R b = R(0), t;"]
    for k in range(forms.shape[0]):
        terms = []
        for j in range(19):
            s = lit(forms[k, j])
            if s is not None:
                terms.append("%s * d[%d]" % (s, j))
        if not terms:
            continue
        lines.append("  t = %s;" % " + ".join(terms))
        lines.append("  b += %s * t * t;" % lit(D[k]))
    lines.append("  return b;")
    lines.append("}")
    return "\n".join(lines)


def emit_beta_x2(name, D, forms):
    """emit_beta on pairs of FP32 data (two characteristic fields), in packed
    FP32: each linear form as in emit_map_x2, then b += D t t."""
    lines = ["__device__ __forceinline__ float2 %s(const float2* d) {" % name,
             "  float2 b = make_float2(0.0f, 0.0f), t;"]
    for k in range(forms.shape[0]):
        terms = [(j, lit(forms[k, j])) for j in range(19)]
        terms = [(j, c) for j, c in terms if c is not None]
        if not terms:
            continue
        for i, (j, c) in enumerate(terms):
            cc = "hw2_pair(%s)" % c[2:-1]
            if i == 0:
                if forms[k, j] == 1:
                    lines.append("  t = d[%d];" % j)
                else:
                    lines.append("  t = __fmul2_rn(%s, d[%d]);" % (cc, j))
            else:
                lines.append("  t = __ffma2_rn(%s, d[%d], t);" % (cc, j))
        if D[k] == 1:
            lines.append("  b = __ffma2_rn(t, t, b);")
        else:
            lines.append("  b = __ffma2_rn(__fmul2_rn(hw2_pair(%s), t), t, b);" % lit(D[k])[2:-1])
    lines.append("  return b;")
    lines.append("}")
    return "\n".join(lines)


def emit_map_T(name, rows):
    lines = ["template <typename R>",
             "__device__ __forceinline__ void %s(const R* l, R* g) {" % name]
    for j in range(19):
        terms = []
        for p, row in enumerate(rows):
            s = lit(row[j])
            if s is not None:
                terms.append("%s * l[%d]" % (s, p))
        if terms:
            lines.append("  g[%d] += %s;" % (j, " + ".join(terms)))
    lines.append("}")
    return "\n".join(lines)


def emit_map_T_x2(name, rows):
    """emit_map_T on pairs of FP32 data (two components), in packed FP32: the
    sum of each row formed as in emit_map_x2, then added to g."""
    lines = ["__device__ __forceinline__ void %s(const float2* l, float2* g) {" % name,
             "  float2 a;"]
    for j in range(19):
        first = True
        for p, row in enumerate(rows):
            s = lit(row[j])
            if s is None:
                continue
            c = "hw2_pair(%s)" % s[2:-1]
            if first:
                lines.append("  a = __fmul2_rn(%s, l[%d]);" % (c, p))
                first = False
            else:
                lines.append("  a = __ffma2_rn(%s, l[%d], a);" % (c, p))
        if not first:
            lines.append("  g[%d] = __fadd2_rn(g[%d], a);" % (j, j))
    lines.append("}")
    return "\n".join(lines)


def emit_beta_grad(name, D, forms):
    lines = ["template <typename R>",
             "__device__ __forceinline__ void %s(const R* d, R s, R* g) {" % name,
             "  R t;"]
    for k in range(forms.shape[0]):
        idx = [(j, lit(forms[k, j])) for j in range(19)]
        idx = [(j, c) for j, c in idx if c is not None]
        if not idx:
            continue
        lines.append("  t = %s * s * (%s);" % (lit(2 * D[k]), " + ".join("%s * d[%d]" % (c, j) for j, c in idx)))
        for j, c in idx:
            lines.append("  g[%d] += %s * t;" % (j, c))
    lines.append("}")
    return "\n".join(lines)


def main_adjoint():
    out = ["// Generated by gen_hweno2d_coef.py (adjoint) from the moment conditions of\n"
           "// Zhao & Qiu, arXiv:2002.08816, Sec. 2.2 Step 5: transposed point maps and\n"
           "// smoothness-indicator gradients.  Do not edit: rerun the generator.\n"
           "#pragma once\n"
           "#include \"hweno2d_coef.cuh\"  // hw2_pair\n"
           "namespace hw2 {"]
    M0 = p0_map()
    MQ = {n: quad_map(n) for n in (1, 2, 3, 4)}
    B4, B2 = gram(4), gram(2)
    for ng in (2, 3):
        pts = points(ng)
        nf = 4 * ng
        out.append("// ---- %d Gauss points per direction" % ng)
        out.append(emit_map_T("p0_faces_ng%d_T" % ng, value_map(M0, 4, pts[:nf])))
        out.append(emit_map_T("p0_interior_ng%d_T" % ng, value_map(M0, 4, pts[nf:])))
        out.append(emit_map_T_x2("p0_faces_ng%d_T_x2" % ng, value_map(M0, 4, pts[:nf])))
        out.append(emit_map_T_x2("p0_interior_ng%d_T_x2" % ng, value_map(M0, 4, pts[nf:])))
        for n in (1, 2, 3, 4):
            out.append(emit_map_T("q%d_faces_ng%d_T" % (n, ng), value_map(MQ[n], 2, pts[:nf])))
    D0, F0 = ldl_forms(B4, M0)
    out.append("// gradients of the smoothness indicators of Eq. (2dGHYZ), dx = dy")
    out.append(emit_beta_grad("beta_p0_grad", D0, F0))
    for n in (1, 2, 3, 4):
        Dn, Fn = ldl_forms(B2, MQ[n])
        out.append(emit_beta_grad("beta_q%d_grad" % n, Dn, Fn))
    out.append("}  // namespace hw2")
    sys.stdout.write("\n\n".join(out) + "\n")


def main():
    out = ["// Generated by gen_hweno2d_coef.py from the moment conditions of Zhao & Qiu,\n"
           "// arXiv:2002.08816, Sec. 2.2 Step 5 (exact rationals, printed to 20 digits).\n"
           "// Do not edit: rerun the generator.\n"
           "#pragma once\n"
           "namespace hw2 {"]
    M0 = p0_map()
    MQ = {n: quad_map(n) for n in (1, 2, 3, 4)}
    B4, B2 = gram(4), gram(2)
    out.append("// a coefficient as a broadcast pair of FP32 values (the packed maps below)\n"
               "__device__ __forceinline__ float2 hw2_pair(double c) {\n"
               "  return make_float2((float)c, (float)c);\n"
               "}")
    for ng in (2, 3):
        pts = points(ng)
        nf = 4 * ng
        out.append("// ---- %d Gauss points per direction: %d interface + %d interior points" %
                   (ng, nf, ng * ng))
        out.append(emit_map("p0_faces_ng%d" % ng, value_map(M0, 4, pts[:nf])))
        out.append(emit_map("p0_interior_ng%d" % ng, value_map(M0, 4, pts[nf:])))
        out.append(emit_map_x2("p0_faces_ng%d_x2" % ng, value_map(M0, 4, pts[:nf])))
        out.append(emit_map_x2("p0_interior_ng%d_x2" % ng, value_map(M0, 4, pts[nf:])))
        for n in (1, 2, 3, 4):
            out.append(emit_map("q%d_faces_ng%d" % (n, ng), value_map(MQ[n], 2, pts[:nf])))
        for n in (1, 2, 3, 4):
            out.append(emit_map_x2("q%d_faces_ng%d_x2" % (n, ng), value_map(MQ[n], 2, pts[:nf])))
    D0, F0 = ldl_forms(B4, M0)
    out.append("// smoothness indicators of Eq. (2dGHYZ), dx = dy")
    out.append(emit_beta("beta_p0", D0, F0))
    for n in (1, 2, 3, 4):
        Dn, Fn = ldl_forms(B2, MQ[n])
        out.append(emit_beta("beta_q%d" % n, Dn, Fn))
    out.append(emit_beta_x2("beta_p0_x2", D0, F0))
    for n in (1, 2, 3, 4):
        Dn, Fn = ldl_forms(B2, MQ[n])
        out.append(emit_beta_x2("beta_q%d_x2" % n, Dn, Fn))
    out.append("}  // namespace hw2")
    sys.stdout.write("\n\n".join(out) + "\n")


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "adjoint":
        main_adjoint()
    else:
        main()
