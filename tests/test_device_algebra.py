"""The device source computes the paper's quantities, checked on the source
text itself with exact (symbolic) arithmetic: the binary64 path
(csrc/eig3_f64.cuh) and, at the end of this file, the compensated binary32
invariants (csrc/eig3_f32c.cuh).

The kernels regroup the paper's formulas into shared products and FMAs
(Algorithms 2, 4 and 5, the trigonometric eigenvalues of Algorithm 6 in
sine form, and the hand-written adjoint).  Here the statements of those device
functions are read from ``csrc/eig3_f64.cuh``, translated to Python and run
on sympy symbols, with fma(a, b, c) = a b + c, the reciprocal exact and the
decimal constants replaced by the exact values they round.  Branches that
only handle the exponent range or exact coalescence (power-of-two scalings,
the cluster mean) are left out; everything else is the text the compiler
sees.  The results must equal the definitions identically:

  I1 = tr A,  J2 = tr(dev(A)^2)/2,  J3 = det dev(A),  Delta = 4 J2^3 - 27 J3^2,
  the gradient = a_I1 dI1/dA + a_J2 dJ2/dA + a_J3 dJ3/dA, with a_J2, a_J3 the
  derivatives of the roots of mu^3 - J2 mu - J3 (divided differences),
  and lambda_k of the sine form the roots of that cubic.
"""
import math
import os
import re
from decimal import Decimal, getcontext

import numpy as np
import pytest

sp = pytest.importorskip("sympy")

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2511_00292_gb300", "csrc")
SRC = os.path.join(CSRC, "eig3_f64.cuh")
SRC_C = os.path.join(CSRC, "eig3_f32c.cuh")

# exact values of the header's constants
EXACT = {
    "kInv3": sp.Rational(1, 3), "kInv6": sp.Rational(1, 6), "kInv9": sp.Rational(1, 9),
    "kInv27": sp.Rational(1, 27), "kHalfSqrt3": sp.sqrt(3) / 2,
    "kTwoOverSqrt3": 2 / sp.sqrt(3), "kK": 2 / (3 * sp.sqrt(3)),
}


class NS:
    """A struct (Inv, Dx, Adj, ...): attributes set by the translated code."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


# ---------------------------------------------------------------------------
# A translator for the C subset of these functions
# ---------------------------------------------------------------------------

def _source(path=None):
    with open(path or SRC) as f:
        return f.read()


def _match(text, i, open_ch, close_ch):
    depth = 0
    for k in range(i, len(text)):
        if text[k] == open_ch:
            depth += 1
        elif text[k] == close_ch:
            depth -= 1
            if depth == 0:
                return k
    raise ValueError("unbalanced")


def _split_top(text, sep):
    parts, depth, cur = [], 0, ""
    for ch in text:
        if ch in "([{":
            depth += 1
        elif ch in ")]}":
            depth -= 1
        if ch == sep and depth == 0:
            parts.append(cur)
            cur = ""
        else:
            cur += ch
    parts.append(cur)
    return parts


def _definition(src, name):
    m = re.search(r"__device__ __forceinline__ [\w:<>]+ " + name + r"\(", src)
    assert m, name
    p0 = m.end() - 1
    p1 = _match(src, p0, "(", ")")
    params = []
    for p in _split_top(src[p0 + 1:p1], ","):
        q = re.search(r"\(&(\w+)\)|&?(\w+)\s*$", p.strip())
        params.append(q.group(1) or q.group(2))
    b0 = src.index("{", p1)
    b1 = _match(src, b0, "{", "}")
    return params, src[b0 + 1:b1]


def _statements(body):
    body = re.sub(r"//[^\n]*", "", body)
    body = "\n".join(l for l in body.split("\n") if not l.strip().startswith("#"))
    out, i, n = [], 0, len(body)
    while i < n:
        while i < n and body[i].isspace():
            i += 1
        if i >= n:
            break
        m = re.match(r"(if|for)\s*\(", body[i:])
        if m:  # control statement: skipped (range scaling, coalescence)
            j = _match(body, i + m.end() - 1, "(", ")") + 1
            while body[j].isspace():
                j += 1
            if body[j] == "{":
                k = _match(body, j, "{", "}") + 1
            else:
                k = j
                depth = 0
                while not (body[k] == ";" and depth == 0):
                    depth += body[k] in "([{"
                    depth -= body[k] in ")]}"
                    k += 1
                k += 1
            out.append(("ctrl", body[i:k]))
            i = k
            continue
        k, depth = i, 0
        while not (body[k] == ";" and depth == 0):
            depth += body[k] in "([{"
            depth -= body[k] in ")]}"
            k += 1
        out.append(("stmt", " ".join(body[i:k].split())))
        i = k + 1
    return out


def _ternaries(e):
    """C conditional expressions c ? a : b (nested, parenthesised or not) as
    Python ((a) if (c) else (b)), outermost first."""
    while "?" in e:
        i = e.index("?")
        start, depth = 0, 0
        for k in range(i - 1, -1, -1):
            if e[k] == ")":
                depth += 1
            elif e[k] == "(":
                if depth == 0:
                    start = k + 1
                    break
                depth -= 1
        end, depth = len(e), 0
        for k in range(i + 1, len(e)):
            if e[k] == "(":
                depth += 1
            elif e[k] == ")":
                if depth == 0:
                    end = k
                    break
                depth -= 1
        grp, q = e[start:end], i - start
        depth, nested, colon = 0, 0, None
        for k in range(q + 1, len(grp)):
            ch = grp[k]
            depth += ch == "("
            depth -= ch == ")"
            if depth == 0 and ch == "?":
                nested += 1
            elif depth == 0 and ch == ":":
                if nested == 0:
                    colon = k
                    break
                nested -= 1
        cond, a, b = grp[:q], grp[q + 1:colon], grp[colon + 1:]
        e = e[:start] + f"(({a}) if ({cond}) else ({b}))" + e[end:]
    return e


def _expr(e, braces="list"):
    if braces == "pair":  # {hi, lo} initialises a compensated pair
        e = e.replace("{", "V2(").replace("}", ")")
    else:
        e = e.replace("{", "[").replace("}", "]")
    e = re.sub(r"(\d+\.\d*(?:e[-+]?\d+)?)f\b", r"\1", e)  # binary32 literals
    e = re.sub(r"dev_scale<\d+>\(\w+\)", "0", e)
    e = re.sub(r"(\w+)<\d+>\(", r"\1(", e)  # sqrt_nonneg<3>( and the like
    e = re.sub(r"(?<![\w.])(\d+\.\d*(?:e[-+]?\d+)?)", lambda m: f"_Q('{m.group(1)}')", e)
    return _ternaries(e)


TYPES = r"(double|int|bool|float|Adj|Adj3|Inv|Eig|Dx|DxShared)"
TYPES_C = r"(int|bool|float|F2|Sum|Grid|Diag|InvC|InvR|Shared|R13|AdjC)"


def _translate(stmt, types=TYPES, ctors=None, braces="list"):
    if stmt.startswith("return "):
        return "__ret__ = " + _expr(stmt[7:], braces)
    m = re.match(r"^(?:const )?" + types + r"\s+(.*)$", stmt)
    if m:
        typ, rest = m.groups()
        if typ in ("int", "bool"):  # exponent tests and coalescence flags: set by the caller
            return ""
        lines = []
        for d in _split_top(rest, ","):
            if "=" not in d:
                lines.append(f"{d.strip()} = {(ctors or {}).get(typ, 'NS()')}")
                continue
            lhs, rhs = d.split("=", 1)
            lines.append(f"{re.sub(r'\[\d+\]', '', lhs.strip())} = {_expr(rhs, braces)}")
        return "\n".join(lines)
    m = re.match(r"^([\w.\[\]]+)\s*=(?!=)\s*(.*)$", stmt)
    if not m:  # a call for its output arguments (the angle): left to the caller
        return ""
    return f"{m.group(1)} = {_expr(m.group(2), braces)}"


def device_function(name, path=None, env=None, types=TYPES, ctors=None, braces="list", **fixed):
    """The device function `name` as a Python callable on sympy values.
    `fixed` binds the names that integer/boolean statements would set."""
    src = _source(path)
    params, body = _definition(src, name)
    # function-like macros of the body become Python functions of the same namespace
    macros = [f"def {m}({a}): return {_expr(b, braces)}" for m, a, b in
              re.findall(r"#define (\w+)\(([^)]*)\)\s+(.*)", body)]
    code = "\n".join(macros + [_translate(s, types, ctors, braces)
                               for kind, s in _statements(body) if kind == "stmt"])

    def fn(*args):
        e = dict(BASE_ENV if env is None else env)
        e.update(fixed)
        e.update(zip(params, args))
        exec(code, e)
        return e.get("__ret__")

    fn.code = code
    return fn


BASE_ENV = dict(
    _Q=sp.Rational, NS=NS, fma=lambda a, b, c: a * b + c, dmul=lambda a, b: a * b,
    recip_pos=lambda x: 1 / x, pow2d=lambda k: sp.Integer(2) ** k,
    times_pow2=lambda x, k: x * sp.Integer(2) ** k, scale2k=lambda x, k: x * sp.Integer(2) ** k,
    **EXACT)
BASE_ENV["dx13"] = lambda *a: device_function("dx13")(*a)


# ---------------------------------------------------------------------------
# Definitions
# ---------------------------------------------------------------------------

def invariants_of(A):
    dev = A - A.trace() / 3 * sp.eye(3)
    J2 = sp.expand((dev * dev).trace() / 2)
    J3 = sp.expand(dev.det())
    return sp.expand(A.trace()), J2, J3


def general_symbols():
    a = sp.symbols("a0:9", real=True)
    return list(a), sp.Matrix(3, 3, a)


def sym_symbols():
    s = sp.symbols("s0:6", real=True)  # (A00, A11, A22, A12, A02, A01)
    A = sp.Matrix([[s[0], s[5], s[4]], [s[5], s[1], s[3]], [s[4], s[3], s[2]]])
    return list(s), A


def zero(expr):
    return sp.expand(expr) == 0


# ---------------------------------------------------------------------------
# Tests
# ---------------------------------------------------------------------------

def test_constants_are_the_nearest_binary64_values():
    src = _source()
    getcontext().prec = 60
    for name, exact in EXACT.items():
        m = re.search(r"constexpr double " + name + r" = ([0-9.e+-]+);", src)
        assert m, name
        assert float(Decimal(m.group(1))) == float(sp.N(exact, 40)), name


def test_invariants_general_source_equals_definitions():
    """Algorithms 1, 2, 4 and 5 as regrouped for the FP64 pipe (shared
    products, FMAs, r1 of dx(A^T) = -r1) are exactly I1, J2, J3 and the
    discriminant."""
    a, A = general_symbols()
    o = device_function("invariants_general")(a)
    I1, J2, J3 = invariants_of(A)
    assert zero(o.I1 - I1)
    assert zero(o.J2 - J2)
    assert zero(o.J3 - J3)
    assert zero(o.D - (4 * J2 ** 3 - 27 * J3 ** 2))


def test_invariants_sym_source_equals_definitions():
    s, A = sym_symbols()
    o = device_function("invariants_sym")(s)
    I1, J2, J3 = invariants_of(A)
    assert zero(o.I1 - I1)
    assert zero(o.J2 - J2)
    assert zero(o.J3 - J3)
    assert zero(o.D - (4 * J2 ** 3 - 27 * J3 ** 2))


def test_delta_terms_carry_the_paper_weights():
    """A plausible slip (a wrong weight of one product group -- the factor
    8 applied as 2^3 to u5, the factor 2 as 2^1 to u13, the 6 of the last
    group -- or r1 of dx(A^T) taken with the wrong sign, or J3's mixed term
    regrouped with the wrong difference) breaks the identities above: the
    checks are not vacuous.  Altering one of them in the translated source
    must fail it."""
    a, A = general_symbols()
    fn = device_function("invariants_general")
    src_code = fn.code
    slips = (("times_pow2(u.r5, 3)", "times_pow2(u.r5, 2)"),
             ("times_pow2(u.r13, 1)", "times_pow2(u.r13, 0)"),
             ("fma(_Q('6.0'),", "fma(_Q('8.0'),"),
             ("dmul(-_Q('9.0'), r1)", "dmul(_Q('9.0'), r1)"))
    for old, _ in slips:
        assert old in src_code, old
    for old, new in slips:
        env = dict(BASE_ENV)
        env["a"] = a
        exec(src_code.replace(old, new, 1), env)
        o = env["__ret__"]
        _, J2, J3 = invariants_of(A)
        assert not zero(o.D - (4 * J2 ** 3 - 27 * J3 ** 2))
    # J3 with e9 for e8 in its mixed term
    assert "fma(t2, dmul(tn, kInv9), s.e8)" in src_code
    env = dict(BASE_ENV)
    env["a"] = a
    exec(src_code.replace("fma(t2, dmul(tn, kInv9), s.e8)", "fma(t2, dmul(tn, kInv9), s.e9)", 1), env)
    _, J2, J3 = invariants_of(A)
    assert not zero(env["__ret__"].J3 - J3)


def _roots_derivatives(r, s1, s2, g):
    """mu_k of the sine form and a_J2 = sum g_k mu_k / p'(mu_k),
    a_J3 = sum g_k / p'(mu_k) for p(mu) = mu^3 - J2 mu - J3."""
    k = EXACT["kK"] * r
    mu = [-k * (s2 + 2 * s1), k * (s1 - s2), k * (2 * s2 + s1)]
    dp = [sp.Mul(*[mu[i] - mu[j] for j in range(3) if j != i]) for i in range(3)]
    aJ3 = sum(g[i] / dp[i] for i in range(3))
    aJ2 = sum(g[i] * mu[i] / dp[i] for i in range(3))
    return mu, aJ2, aJ3


def test_adjoint_scalars_source_are_root_derivatives():
    """a_J2 2^k and a_J3 2^2k (divided differences over the gaps (2r/sqrt3)
    sigma, r = m 2^k; here k = 0) are the derivatives of the roots of the
    depressed cubic, weighted by g."""
    r, s1, s2 = sp.symbols("r sigma1 sigma2", positive=True)
    g = sp.symbols("g1:4", real=True)
    o = device_function("adjoint_scalars", z1=False, z2=False, rz=False, kr=0)(
        r, s1, s2, *g)
    _, aJ2, aJ3 = _roots_derivatives(r, s1, s2, g)
    assert sp.simplify(o.aJ3s - aJ3) == 0
    assert sp.simplify(o.aJ2s - aJ2) == 0
    assert sp.simplify(o.aI1 - sum(g) / 3) == 0
    assert o.k == 0 and o.rz is False


def test_sine_form_eigenvalues_are_the_cubic_roots():
    """lambda_k = I1/3 + mu_k of the source's sine form are the roots of
    lambda^3 - I1 lambda^2 + ... for J2 = r^2/3 and J3 = (2 r^3/27) cos(3 psi)
    with sigma1 = sin psi, sigma2 = sin(pi/3 - psi), and they ascend."""
    I1, r, s1, s2 = sp.symbols("I1 r sigma1 sigma2", real=True)
    fn = device_function("eigvals_from_inv")
    code = "\n".join(l for l in fn.code.split("\n")
                     if not re.match(r"\s*(o\.(j2_clamped|d_clamped|r) =|J2p|Dp|triple_angle_sines)", l))
    env = dict(BASE_ENV)
    env["v"] = NS(I1=I1)
    env["o"] = NS(r=r, sigma1=s1, sigma2=s2)
    exec(code.replace("o = NS()", ""), env)
    o = env["__ret__"]
    lam = [o.l1, o.l2, o.l3]
    assert zero(sum(lam) - I1)
    assert zero(lam[1] - lam[0] - 2 * r / sp.sqrt(3) * s1)     # gaps (2r/sqrt3) sigma
    assert zero(lam[2] - lam[1] - 2 * r / sp.sqrt(3) * s2)
    for psi in (0.0, 0.1, 0.37, math.pi / 6):
        sub = {I1: sp.Rational(7, 5), r: sp.Rational(3, 2),
               s1: sp.sin(sp.nsimplify(psi)), s2: sp.sin(sp.pi / 3 - sp.nsimplify(psi))}
        J2 = sub[r] ** 2 / 3
        J3 = 2 * sub[r] ** 3 / 27 * sp.cos(3 * sp.nsimplify(psi))
        for lk in lam:
            mu = lk.subs(sub) - sub[I1] / 3
            assert abs(sp.N(mu ** 3 - J2 * mu - J3, 50)) < 1e-40


def test_grad_general_source_is_the_chain_rule():
    """G = a_I1 dI1/dA + a_J2 dJ2/dA + a_J3 dJ3/dA (the scalars at k = 0,
    where the exact power-of-two unit changes leave them as they are)."""
    a, A = general_symbols()
    aI1, b2, b3 = sp.symbols("aI1 aJ2 aJ3", real=True)
    G = [None] * 9
    device_function("grad_general")(a, NS(aI1=aI1, aJ2s=b2, aJ3s=b3, k=0, rz=False), G)
    I1, J2, J3 = invariants_of(A)
    for idx in range(9):
        want = aI1 * sp.diff(I1, a[idx]) + b2 * sp.diff(J2, a[idx]) + b3 * sp.diff(J3, a[idx])
        assert zero(G[idx] - want), idx


def test_grad_sym_source_is_the_chain_rule():
    """The symmetric gradient is with respect to the six stored entries
    (off-diagonal: G_ij + G_ji)."""
    s, A = sym_symbols()
    aI1, b2, b3 = sp.symbols("aI1 aJ2 aJ3", real=True)
    G = [None] * 6
    device_function("grad_sym")(s, NS(aI1=aI1, aJ2s=b2, aJ3s=b3, k=0, rz=False), G)
    I1, J2, J3 = invariants_of(A)
    for idx in range(6):
        want = aI1 * sp.diff(I1, s[idx]) + b2 * sp.diff(J2, s[idx]) + b3 * sp.diff(J3, s[idx])
        assert zero(G[idx] - want), idx


def test_fused_adjoint_scalars_are_root_derivatives():
    """adjoint_vjp (k = 0, no coalescence): a_J2 and a_J3 are the weighted
    derivatives of the roots of the depressed cubic, from the forward's m,
    kK m and 2 sigma1 + sigma2, with Rh = 1 / (3 kK m P) from recip3_pos; and
    a_I1 = g2 + n2 / 3 is the mean weight."""
    r, s1, s2 = sp.symbols("r sigma1 sigma2", positive=True)
    g = sp.symbols("g1:4", real=True)
    env = dict(BASE_ENV, recip3_pos=lambda x: 1 / (3 * x), hi_abs=lambda x: 0)
    fn = device_function("adjoint_vjp", env=env, z1=False, z2=False, rz=False)
    f = NS(e=NS(sigma1=s1, sigma2=s2), m=r, kKm=EXACT["kK"] * r, c12=2 * s1 + s2, kr=0)
    o = fn(f, *g)
    _, aJ2, aJ3 = _roots_derivatives(r, s1, s2, g)
    assert sp.simplify(o.aJ3s - aJ3) == 0
    assert sp.simplify(o.aJ2s - aJ2) == 0
    assert sp.simplify(o.g2 + o.n2 / 3 - sum(g) / 3) == 0


def _struct_fields(name):
    body = re.search(r"struct " + name + r" \{(.*?)\};", _source(), re.S).group(1)
    body = re.sub(r"//[^\n]*", "", body)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            out += [f.strip() for f in re.sub(r"^\w+\s+", "", decl).split(",")]
    return out


def _shared_of(inv_name, struct, args):
    """Run the invariants function's source and build the products it hands
    on to the fused kernel from its own `*x = Struct{...}` initializer."""
    fn = device_function(inv_name)
    env = dict(BASE_ENV)
    params, body = _definition(_source(), inv_name)
    env.update(zip(params, args))
    exec(fn.code, env)
    init = re.search(r"\*x = " + struct + r"\{(.*?)\};", body, re.S).group(1)
    vals = [eval(_expr(e.strip()), env) for e in _split_top(init, ",")]
    fields = _struct_fields(struct)
    assert len(vals) == len(fields)
    return NS(**dict(zip(fields, vals))), env["__ret__"]


def _fused_grad(name, x, J2, aI1, b2, b3, n):
    fn = device_function(name)
    code = fn.code.replace("b2 = NS()", "b2 = s.aJ2s").replace("b3 = NS()", "b3 = s.aJ3s")
    G = [None] * n
    env = dict(BASE_ENV)
    g2 = sp.Symbol("g2_weight", real=True)
    env.update(x=x, J2=J2, s=NS(n2=3 * aI1 - 3 * g2, g2=g2, aJ2s=b2, aJ3s=b3, k=0, rz=False),
               G=G)
    exec(code, env)
    return [sp.expand(gi) for gi in G]


def test_fused_grad_general_source_is_the_chain_rule():
    """The fused kernel's gradient (grad_general_vjp, at k = 0: the scalings
    are the identity) on the products invariants_general hands on is
    a_I1 dI1/dA + a_J2 dJ2/dA + a_J3 dJ3/dA, entry by entry."""
    a, A = general_symbols()
    aI1, b2, b3 = sp.symbols("aI1 aJ2 aJ3", real=True)
    x, inv = _shared_of("invariants_general", "ShareG", [a])
    G = _fused_grad("grad_general_vjp", x, inv.J2, aI1, b2, b3, 9)
    I1, J2, J3 = invariants_of(A)
    assert zero(inv.J2 - J2)
    for idx in range(9):
        want = aI1 * sp.diff(I1, a[idx]) + b2 * sp.diff(J2, a[idx]) + b3 * sp.diff(J3, a[idx])
        assert zero(G[idx] - want), idx


def test_fused_grad_sym_source_is_the_chain_rule():
    s6, A = sym_symbols()
    aI1, b2, b3 = sp.symbols("aI1 aJ2 aJ3", real=True)
    x, inv = _shared_of("invariants_sym", "ShareS", [s6])
    G = _fused_grad("grad_sym_vjp", x, inv.J2, aI1, b2, b3, 6)
    I1, J2, J3 = invariants_of(A)
    for idx in range(6):
        want = aI1 * sp.diff(I1, s6[idx]) + b2 * sp.diff(J2, s6[idx]) + b3 * sp.diff(J3, s6[idx])
        assert zero(G[idx] - want), idx


def test_fused_grad_check_sees_a_slip():
    """A transposed operand in the shared bracket breaks the identity above."""
    a, A = general_symbols()
    aI1, b2, b3 = sp.symbols("aI1 aJ2 aJ3", real=True)
    x, inv = _shared_of("invariants_general", "ShareG", [a])
    fn = device_function("grad_general_vjp")
    code = fn.code.replace("b2 = NS()", "b2 = s.aJ2s").replace("b3 = NS()", "b3 = s.aJ3s")
    old = "G[1] = fma(D[3], q8, dmul(b3, P[1]))"
    assert old in code
    G = [None] * 9
    env = dict(BASE_ENV)
    env.update(x=x, J2=inv.J2, s=NS(n2=3 * aI1, g2=0, aJ2s=b2, aJ3s=b3, k=0, rz=False), G=G)
    exec(code.replace(old, "G[1] = fma(D[1], q8, dmul(b3, P[1]))"), env)
    I1, J2, J3 = invariants_of(A)
    want = aI1 * sp.diff(I1, a[1]) + b2 * sp.diff(J2, a[1]) + b3 * sp.diff(J3, a[1])
    assert not zero(G[1] - want)


# ---------------------------------------------------------------------------
# The compensated binary32 source (csrc/eig3_f32c.cuh) in exact arithmetic
# ---------------------------------------------------------------------------
#
# TwoSum and TwoProduct are error-free, so in exact arithmetic every low part
# is zero and a compensated pair or Sum2 state is its value; the terms the
# kernels drop (the low-by-low products) vanish with them.  The compensated
# invariants must then be the definitions exactly (times 6 and 27, at scale 1).

class V:
    """A compensated pair (h, l) or Sum2 state (s, c), exactly: its value."""

    def __init__(self, v):
        self.v = sp.sympify(v)

    h = property(lambda self: self.v)
    s = property(lambda self: self.v)
    l = property(lambda self: sp.Integer(0))
    c = property(lambda self: sp.Integer(0))

    def __add__(self, o):
        return V(self.v + val(o))

    def __sub__(self, o):
        return V(self.v - val(o))

    def __neg__(self):
        return V(-self.v)


def val(x):
    return x.v if isinstance(x, V) else x


ENV_C = dict(
    _Q=sp.Rational, NS=NS, V2=lambda a, b: V(val(a) + val(b)),
    two_sum=lambda a, b: V(val(a) + val(b)), two_prod=lambda a, b: V(val(a) * val(b)),
    mul=lambda x, y: V(val(x) * val(y)), neg=lambda x: V(-val(x)),
    scale2=lambda x, p: V(val(x) * val(p)), start=lambda x: V(val(x)),
    pair=lambda x: V(val(x)), sq=lambda x: V(val(x) ** 2), done=lambda x: V(val(x)),
    gstart=lambda x, y: V(val(x) * val(y)), gadd=lambda g, x, y: V(val(g) + val(x) * val(y)),
    gsum=val, gdiff=lambda x, y: V(val(x) - val(y)),
    round1=val, __fmul_rn=lambda a, b: val(a) * val(b), __fadd_rn=lambda a, b: val(a) + val(b),
    __fsub_rn=lambda a, b: val(a) - val(b), __fmaf_rn=lambda a, b, c: val(a) * val(b) + val(c),
    __fdividef=lambda a, b: val(a) / val(b),
    fmaf=lambda a, b, c: a * b + c, det2=lambda a, d, b, c: a * d - b * c,
    pow2_from_field=lambda f: 1, **EXACT)
# decimal constants of the binary32 source and the exact values they round
LITERALS_C = {"1.15470053837925152902": "kTwoOverSqrt3",
              "0.38490017945975050967": "kK",
              "0.86602540378443864676": "kHalfSqrt3"}
CTORS_C = {"R13": "NS(r=[None] * 13)"}


def f32c_function(name, **fixed):
    fixed.setdefault("E", 127)  # E = 127: the scale 2^(127 - E) is 1
    fn = device_function(name, path=SRC_C, env=ENV_C, types=TYPES_C, ctors=CTORS_C,
                         braces="pair", **fixed)
    code = fn.code
    for lit, name_ in LITERALS_C.items():
        code = code.replace(f"_Q('{lit}')", name_)
    params, _ = _definition(_source(SRC_C), name)

    def run(*args):
        e = dict(ENV_C)
        e.update(fixed)
        e.update(zip(params, args))
        exec(code, e)
        return e.get("__ret__")

    run.code = code
    return run


ENV_C["diag_parts"] = lambda *a: f32c_function("diag_parts")(*a)
ENV_C["dx_c"] = lambda *a: f32c_function("dx_c")(*a)
ENV_C["sq1"] = lambda r: val(r) ** 2
ENV_C["disc_sym_compensated"] = lambda *a: f32c_function("disc_sym_compensated")(*a)
ENV_C["disc_sym_rounded"] = lambda *a: f32c_function("disc_sym_rounded")(*a)


def _check_scaled_invariants(o, A):
    I1, J2, J3 = invariants_of(A)
    assert o.e == 0
    assert zero(val(o.I1) - I1)
    assert zero(val(o.J2x6) - 6 * J2)
    assert zero(val(o.J3x27) - 27 * J3)
    assert zero(val(o.D) - (4 * J2 ** 3 - 27 * J3 ** 2))


@pytest.mark.parametrize("eig", [False, True])
def test_compensated_invariants_sym_source_equals_definitions(eig):
    """The symmetric compensated invariants (Algorithms 1, 2, 4, 5 with the
    symmetric identities and reading R1, every r_i summed term by term) are
    I1, 6 J2, 27 J3 and the discriminant exactly -- with the discriminant
    finished either way (compensated for the invariants output, the rounded
    non-negative sum for the eigenvalue kernels)."""
    s6, A = sym_symbols()
    _check_scaled_invariants(f32c_function("invariants_sym_c", EIG=eig)(*s6), A)


def test_grid_invariants_sym_source_equals_definitions():
    """The symmetric invariants of the eigenvalue kernels (every sum on its
    fixed grid, Delta from the rounded r_i with -r12 for r12) are I1, 6 J2,
    27 J3 and the discriminant exactly."""
    s6, A = sym_symbols()
    _check_scaled_invariants(f32c_function("invariants_sym_eig")(*s6), A)


@pytest.mark.parametrize("old,new", [
    ("gadd(j3, mul(bb, t2), _Q('9.0'))", "gadd(j3, mul(bb, t2), _Q('8.0'))"),
    ("gadd(gadd(s89, aa, c), neg(ab), d1)", "gadd(s89, aa, c)"),
    ("gdiff(g13, g12n)", "gdiff(g13, g12n) + r13"),
    ("gadd(j2, cc, _Q('6.0'))", "gadd(j2, cc, _Q('3.0'))"),
    ("__fmul_rn(r14, r14)", "_Q('0.0')"),
    ("gadd(s1213, neg(ac), d0)", "gadd(s1213, ac, d0)"),
])
def test_grid_invariants_sym_check_sees_a_slip(old, new):
    """A wrong weight, a dropped term or a flipped sign in the grid form
    breaks one of the identities above."""
    s6, A = sym_symbols()
    fn = f32c_function("invariants_sym_eig")
    assert old in fn.code
    e = dict(ENV_C)
    e.update(E=127)
    e.update(zip(["a00", "a11", "a22", "c0", "b0", "a0"], s6))
    exec(fn.code.replace(old, new, 1), e)
    o = e["__ret__"]
    I1, J2, J3 = invariants_of(A)
    assert not (zero(val(o.J2x6) - 6 * J2) and zero(val(o.J3x27) - 27 * J3)
                and zero(val(o.D) - (4 * J2 ** 3 - 27 * J3 ** 2)))


def test_rounded_discriminant_keeps_the_weights():
    """A wrong weight in the rounded form (2 for 14, or a dropped r14^2)
    breaks the identity: the check above is not vacuous for it."""
    s6, A = sym_symbols()
    fn = f32c_function("disc_sym_rounded")
    code = fn.code
    for old, new in (("_Q('14.0')", "_Q('2.0')"), ("sq1(r14)", "_Q('0.0')")):
        assert old in code
    r = sp.symbols("r2 r3 r4 r8 r9 r10 r11 r12 r13 r14")
    want = 14 * (r[0] ** 2 + r[1] ** 2 + r[2] ** 2) + 2 * sum(x ** 2 for x in r[3:9]) + r[9] ** 2
    assert zero(val(fn(*r)) - want)
    for old, new in (("_Q('14.0')", "_Q('2.0')"), ("sq1(r14)", "_Q('0.0')")):
        e = dict(ENV_C)
        e.update(zip(["r2", "r3", "r4", "r8", "r9", "r10", "r11", "r12", "r13", "r14"], r))
        exec(code.replace(old, new, 1), e)
        assert not zero(val(e["__ret__"]) - want)


def test_compensated_invariants_general_source_equals_definitions():
    """The general compensated invariants, with dx(A) and dx(A^T) from the
    same term-by-term dx_c, are I1, 6 J2, 27 J3 and the discriminant exactly."""
    a, A = general_symbols()
    _check_scaled_invariants(f32c_function("invariants_general_c")(a), A)


def test_binary32_constants_are_the_nearest_values():
    src = _source(SRC_C)
    for lit, name in LITERALS_C.items():
        assert lit + "f" in src
        assert np.float32(float(lit)) == np.float32(float(sp.N(EXACT[name], 30)))


def test_compensated_adjoint_scalars_are_root_derivatives():
    """r a_J2 and r^2 a_J3 of the binary32 adjoint (its divided differences
    over the gaps (2/sqrt3) r sigma) are the weighted derivatives of the roots
    of the depressed cubic; checked at exact rational points (the source's
    range test on r needs a number)."""
    fn = f32c_function("adjoint_c", z1=False, z2=False)
    for r, s1, s2, g in ((sp.Rational(3, 2), sp.Rational(1, 5), sp.Rational(2, 3),
                          (sp.Rational(1, 7), sp.Rational(-2, 3), sp.Rational(5, 4))),
                         (sp.Rational(7, 100), sp.Rational(1, 1000), sp.Rational(7, 8),
                          (sp.Integer(2), sp.Integer(-1), sp.Rational(1, 3)))):
        o = fn(r, s1, s2, *g)
        _, aJ2, aJ3 = _roots_derivatives(r, s1, s2, g)
        assert sp.simplify(o.aJ3r2 - r ** 2 * aJ3) == 0
        assert sp.simplify(o.aJ2r - r * aJ2) == 0
        assert sp.simplify(o.aI1 - sum(g) / 3) == 0
        assert o.inv_r == 1 / r


@pytest.mark.parametrize("layout", ["general9", "sym6"])
def test_compensated_gradients_are_the_chain_rule(layout):
    """The binary32 gradients (dev(A)/r, Kahan 2x2 cofactors, the adjoint's
    scalars in units of r) are the chain rule through I1, J2, J3."""
    if layout == "general9":
        x, A = general_symbols()
        name, n = "grad_general_c", 9
    else:
        x, A = sym_symbols()
        name, n = "grad_sym_c", 6
    aI1, b2, b3, ir = sp.symbols("aI1 aJ2r aJ3r2 ir", real=True)
    G = [None] * n
    f32c_function(name)(x, NS(aI1=aI1, aJ2r=b2, aJ3r2=b3, inv_r=ir), G)
    I1, J2, J3 = invariants_of(A)
    for idx in range(n):
        want = aI1 * sp.diff(I1, x[idx]) + b2 * ir * sp.diff(J2, x[idx]) + \
            b3 * ir ** 2 * sp.diff(J3, x[idx])
        assert zero(val(G[idx]) - want), idx
