"""The 2D coefficient tables the CUDA kernels compile in
(csrc/hweno2d_coef.cuh, generated in exact arithmetic by sympy) against the
oracle's own numerical derivation of the same moment conditions (a KKT solve
in FP64).  The two derivations share no code; this compares their outputs."""

import os
import re

import numpy as np
import pytest

from oracle import oracle as O

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2002_08816_gb300", "csrc", "hweno2d_coef.cuh")


def _parse():
    txt = open(HDR).read()
    maps, betas = {}, {}
    for m in re.finditer(r"void (\w+)\(const R\* d, R\* o\) \{(.*?)\n\}", txt, re.S):
        rows = {}
        for line in m.group(2).strip().splitlines():
            mm = re.match(r"\s*o\[(\d+)\] = (.*);", line)
            coef = {int(j): float(c) for c, j in re.findall(r"R\(([-0-9.eE+]+)\) \* d\[(\d+)\]", mm.group(2))}
            rows[int(mm.group(1))] = coef
        maps[m.group(1)] = rows
    for m in re.finditer(r"R (beta_\w+)\(const R\* d\) \{(.*?)\n\}", txt, re.S):
        terms, cur = [], None
        for line in m.group(2).splitlines():
            if line.strip().startswith("t ="):
                cur = {int(j): float(c) for c, j in re.findall(r"R\(([-0-9.eE+]+)\) \* d\[(\d+)\]", line)}
            elif line.strip().startswith("b +="):
                w = float(re.search(r"R\(([-0-9.eE+]+)\)", line).group(1))
                terms.append((w, cur))
        betas[m.group(1)] = terms
    return maps, betas


MAPS, BETAS = _parse()


def _apply(rows, d):
    return np.array([sum(c * d[j] for j, c in rows[p].items()) for p in range(len(rows))])


def _split(d):
    ub = d[:9]
    vb = np.zeros(9)
    wb = np.zeros(9)
    for k, cell in enumerate([2, 4, 5, 6, 8]):
        vb[cell - 1] = d[9 + k]
        wb[cell - 1] = d[14 + k]
    return ub, vb, wb


@pytest.mark.parametrize("ng", [2, 3])
def test_generated_maps_match_the_oracle(ng):
    rng = np.random.default_rng(ng)
    nf = 4 * ng
    for _ in range(6):
        d = rng.normal(size=19)
        val, beta = O.recon_candidates2d(*_split(d), ng)
        np.testing.assert_allclose(_apply(MAPS["p0_faces_ng%d" % ng], d), val[0, :nf], atol=1e-12)
        np.testing.assert_allclose(_apply(MAPS["p0_interior_ng%d" % ng], d), val[0, nf:], atol=1e-12)
        for n in (1, 2, 3, 4):
            np.testing.assert_allclose(_apply(MAPS["q%d_faces_ng%d" % (n, ng)], d), val[n, :nf],
                                       atol=1e-12)
        got = [sum(w * sum(c * d[j] for j, c in f.items()) ** 2 for w, f in BETAS[name])
               for name in ("beta_p0", "beta_q1", "beta_q2", "beta_q3", "beta_q4")]
        np.testing.assert_allclose(got, beta, rtol=1e-11)


def _parse_x2():
    """The packed (two components at once) copies of the p0 maps: {name of
    the scalar map: {point: {datum: coefficient}}}."""
    txt = open(HDR).read()
    maps = {}
    for m in re.finditer(r"void (\w+)_x2\(const float2\* d, float2\* o\) \{(.*?)\n\}", txt, re.S):
        rows, cur = {}, {}
        for line in m.group(2).splitlines():
            t = re.match(r"\s*a = __f(?:mul|fma)2_rn\(hw2_pair\(([-0-9.eE+]+)\), d\[(\d+)\]", line)
            if t:
                cur[int(t.group(2))] = float(t.group(1))
                continue
            o = re.match(r"\s*o\[(\d+)\] = a;", line)
            if o:
                rows[int(o.group(1))] = cur
                cur = {}
        maps[m.group(1)] = rows
    return maps


def test_packed_maps_are_the_scalar_maps():
    x2 = _parse_x2()
    names = {"p0_faces_ng2", "p0_interior_ng2", "p0_faces_ng3", "p0_interior_ng3"}
    names |= {"q%d_faces_ng%d" % (n, ng) for n in (1, 2, 3, 4) for ng in (2, 3)}
    assert set(x2) == names
    for name, rows in x2.items():
        assert rows == MAPS[name], name


def test_packed_smoothness_indicators_are_the_scalar_ones():
    """beta_*_x2 (two characteristic fields at once) hold the weights and
    linear forms of the scalar indicators, in the same order."""
    txt = open(HDR).read()
    packed = {}
    for m in re.finditer(r"float2 (beta_\w+)_x2\(const float2\* d\) \{(.*?)\n\}", txt, re.S):
        terms, cur = [], {}
        for line in m.group(2).splitlines():
            t0 = re.match(r"\s*t = d\[(\d+)\];", line)
            t = re.match(r"\s*t = __f(?:mul|fma)2_rn\(hw2_pair\(([-0-9.eE+]+)\), d\[(\d+)\]", line)
            if t0:
                cur = {int(t0.group(1)): 1.0}
            elif t:
                if "__fmul2_rn" in line:
                    cur = {}
                cur[int(t.group(2))] = float(t.group(1))
            elif re.match(r"\s*b = __ffma2_rn\(t, t, b\);", line):
                terms.append((1.0, cur))
            else:
                w = re.match(r"\s*b = __ffma2_rn\(__fmul2_rn\(hw2_pair\(([-0-9.eE+]+)\), t\), t, b\);", line)
                if w:
                    terms.append((float(w.group(1)), cur))
        packed[m.group(1)] = terms
    assert set(packed) == set(BETAS) == {"beta_p0", "beta_q1", "beta_q2", "beta_q3", "beta_q4"}
    for name in BETAS:
        assert packed[name] == BETAS[name], name


ADJ = os.path.join(os.path.dirname(HDR), "hweno2d_adj_coef.cuh")


def test_packed_transposes_are_the_scalar_transposes():
    """The adjoint's packed transposed p0 maps hold the coefficients of its
    scalar ones (which the GPU adjoint tests hold to the oracle's gradient)."""
    txt = open(ADJ).read()
    scalar, packed = {}, {}
    for m in re.finditer(r"void (p0_\w+_T)\(const R\* l, R\* g\) \{(.*?)\n\}", txt, re.S):
        rows = {}
        for line in m.group(2).strip().splitlines():
            mm = re.match(r"\s*g\[(\d+)\] \+= (.*);", line)
            rows[int(mm.group(1))] = {int(p): float(c) for c, p in
                                      re.findall(r"R\(([-0-9.eE+]+)\) \* l\[(\d+)\]", mm.group(2))}
        scalar[m.group(1)] = rows
    for m in re.finditer(r"void (p0_\w+_T)_x2\(const float2\* l, float2\* g\) \{(.*?)\n\}", txt, re.S):
        rows, cur = {}, {}
        for line in m.group(2).splitlines():
            t = re.match(r"\s*a = __f(?:mul|fma)2_rn\(hw2_pair\(([-0-9.eE+]+)\), l\[(\d+)\]", line)
            if t:
                cur[int(t.group(2))] = float(t.group(1))
                continue
            o = re.match(r"\s*g\[(\d+)\] = __fadd2_rn\(g\[\d+\], a\);", line)
            if o:
                rows[int(o.group(1))] = cur
                cur = {}
        packed[m.group(1)] = rows
    assert set(packed) == set(scalar) == {"p0_faces_ng2_T", "p0_interior_ng2_T",
                                          "p0_faces_ng3_T", "p0_interior_ng3_T"}
    for name in scalar:
        assert packed[name] == scalar[name], name
