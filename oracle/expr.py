"""Oracle (test infrastructure): the general stencil.apply, evaluated plainly.

Section 2.2 of the paper: a stencil.apply reads its input temps at constant
offsets and yields one value per point of its output's bounds; its body is
arbitrary arithmetic on those reads (Section 4.1's Piacsek-Williams
advection is such a body: products of sums of neighbours).  This module
evaluates a body given as an expression string -- the grammar the library's
stencil_apply_expr takes -- over whole arrays with numpy, one IEEE binary64
operation per operator of the expression, in the order of its tree
(left-associative + - and * /, * and / binding tighter, unary minus), so
every output is the expression's binary64 value.

Only tests/, smoke() and bench.py's CPU baseline use the oracle; the
library never does.  Pins: tests/test_oracle_expr.py (closed forms on
integer fields, equality with oracle.apply_linear for linear bodies and
with oracle.advect_uvw for the advection written as expressions).
"""
import re

import numpy as np

_TOKEN = re.compile(r"""\s*(?:
    (?P<ref>a(?P<idx>[0-9])\s*\(\s*(?P<dx>[+-]?[0-9]+)\s*,\s*(?P<dy>[+-]?[0-9]+)\s*,\s*(?P<dz>[+-]?[0-9]+)\s*\))
  | (?P<num>(?:[0-9]+\.?[0-9]*|\.[0-9]+)(?:[eE][+-]?[0-9]+)?)
  | (?P<op>[-+*/()])
)""", re.VERBOSE)


def _tokens(expr):
    pos, out = 0, []
    text = expr.rstrip()
    while pos < len(text):
        m = _TOKEN.match(text, pos)
        if not m or m.end() == pos:
            raise ValueError(f"cannot read the expression at offset {pos}")
        pos = m.end()
        if m.group("ref"):
            d = tuple(int(m.group(k)) for k in ("dx", "dy", "dz"))
            out.append(("ref", int(m.group("idx")), d))
        elif m.group("num"):
            v = float(m.group("num"))
            if not np.isfinite(v):
                raise ValueError("number out of range")
            out.append(("num", v))
        else:
            out.append(("op", m.group("op")))
    return out


class _Parser:
    """Builds the expression tree: ('num', v), ('ref', n, (dx, dy, dz)),
    ('neg', t), (op, left, right)."""

    def __init__(self, toks):
        self.t, self.i = toks, 0

    def peek(self):
        return self.t[self.i] if self.i < len(self.t) else None

    def take(self):
        tok = self.peek()
        if tok is None:
            raise ValueError("the expression ends too early")
        self.i += 1
        return tok

    def expr(self):
        node = self.term()
        while self.peek() in (("op", "+"), ("op", "-")):
            op = self.take()[1]
            node = (op, node, self.term())
        return node

    def term(self):
        node = self.unary()
        while self.peek() in (("op", "*"), ("op", "/")):
            op = self.take()[1]
            node = (op, node, self.unary())
        return node

    def unary(self):
        if self.peek() == ("op", "-"):
            self.take()
            return ("neg", self.unary())
        return self.primary()

    def primary(self):
        tok = self.take()
        if tok == ("op", "("):
            node = self.expr()
            if self.take() != ("op", ")"):
                raise ValueError("expected ')'")
            return node
        if tok[0] in ("num", "ref"):
            return tok
        raise ValueError(f"unexpected {tok}")


def parse(expr, ninputs):
    """The expression's tree and its radius r = max(1, largest |offset|)."""
    p = _Parser(_tokens(expr))
    tree = p.expr()
    if p.peek() is not None:
        raise ValueError("unexpected text after the expression")
    radius = 1

    def check(node):
        nonlocal radius
        if node[0] == "ref":
            if node[1] >= ninputs:
                raise ValueError("input index beyond the inputs given")
            for d in node[2]:
                if abs(d) > 3:
                    raise ValueError("offset beyond three cells")
                radius = max(radius, abs(d))
        elif node[0] == "neg":
            check(node[1])
        elif node[0] in "+-*/":
            check(node[1])
            check(node[2])

    check(tree)
    return tree, radius


def apply_expr(inputs, expr, out=None):
    """out(x) = expr for every point x with r <= index <= n + 1 - r on each
    axis (arrays indexed [z, y, x] with a one-cell halo, as everywhere in the
    oracle); the other points of out keep their values (a copy of `out`, or
    zeros)."""
    inputs = [np.asarray(a, dtype=np.float64) for a in inputs]
    shape = inputs[0].shape
    if any(a.shape != shape for a in inputs):
        raise ValueError("inputs of different shapes")
    tree, r = parse(expr, len(inputs))
    res = np.zeros(shape) if out is None else np.array(out, dtype=np.float64, copy=True)
    nz2, ny2, nx2 = shape
    if min(nz2, ny2, nx2) - 2 * r < 1:
        return res

    def view(n, d):
        dx, dy, dz = d
        return inputs[n][r + dz:nz2 - r + dz, r + dy:ny2 - r + dy, r + dx:nx2 - r + dx]

    def ev(node):
        kind = node[0]
        if kind == "num":
            return np.float64(node[1])
        if kind == "ref":
            return view(node[1], node[2])
        if kind == "neg":
            return np.negative(ev(node[1]))
        a, b = ev(node[1]), ev(node[2])
        return {"+": np.add, "-": np.subtract, "*": np.multiply, "/": np.divide}[kind](a, b)

    val = ev(tree)
    res[r:nz2 - r, r:ny2 - r, r:nx2 - r] = np.broadcast_to(val, res[r:nz2 - r, r:ny2 - r, r:nx2 - r].shape)
    return res
