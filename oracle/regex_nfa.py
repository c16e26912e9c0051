"""Regular expression -> epsilon-free NFA, for the CPU oracle.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the GPU library (whose compiler builds a minimised DFA by a different route).

The paper states queries as regular expressions over labels and inverse
labels (section 2: 2-NFA and 2-RPQ definitions; section 5.2: SPARQL paths are
turned into automata).  It fixes no concrete syntax, so the query syntax is:

    alt  := seq ('|' seq)*
    seq  := post ([/ . whitespace] post)*      (juxtaposition also concatenates)
    post := atom ('*' | '+' | '?')*
    atom := LABEL | '^' atom | '(' alt ')'
    LABEL := decimal label id in [0, L)

``^R`` is the inverse language R^- of section 4 (single-destination part):
every word reversed and every symbol inverted, so ``^^a = a`` (section 2:
(a^-)^- = a).  Symbols are ints: ``a`` in [0, L) is a forward label and
``a + L`` is a^-.

Construction: Thompson's construction (Thompson 1968) into an automaton with
epsilon moves, where the inverse of a fragment is that fragment with every
edge reversed, every symbol inverted and start/end swapped; then epsilon
moves are removed by closure, giving the transition-labelled 2-NFA of
section 2 (states Q, transitions with labels, start set Q_S, final set Q_F).
"""

from __future__ import annotations

from dataclasses import dataclass, field


class RegexError(ValueError):
    pass


@dataclass
class Nfa:
    """epsilon-free 2-NFA: transitions (q, a, q') with a in [0, 2L)."""

    n_states: int
    n_labels: int
    transitions: list  # list of (from, symbol, to)
    starts: list
    finals: list

    def delta(self):
        d = {}
        for q, a, r in self.transitions:
            d.setdefault((q, a), set()).add(r)
        return d

    def accepts(self, word) -> bool:
        """Subset simulation of the automaton on a word of symbols."""
        d = self.delta()
        cur = set(self.starts)
        for a in word:
            nxt = set()
            for q in cur:
                nxt |= d.get((q, a), set())
            cur = nxt
            if not cur:
                return False
        return bool(cur & set(self.finals))

    def arrays(self):
        """(S, t_from, t_label, t_to, starts, finals) as plain int lists."""
        tf = [t[0] for t in self.transitions]
        tl = [t[1] for t in self.transitions]
        tt = [t[2] for t in self.transitions]
        return self.n_states, tf, tl, tt, list(self.starts), list(self.finals)


# ------------------------------------------------------------------ parser --

def _tokenize(text: str):
    toks = []
    i = 0
    while i < len(text):
        c = text[i]
        if c.isdigit():
            j = i
            while j < len(text) and text[j].isdigit():
                j += 1
            toks.append(("LABEL", int(text[i:j])))
            i = j
        elif c in "|*+?^()":
            toks.append((c, None))
            i += 1
        elif c in "/·." :
            toks.append(("CAT", None))
            i += 1
        elif c.isspace():
            toks.append(("WS", None))
            i += 1
        else:
            raise RegexError(f"unexpected character {c!r} at {i}")
    # whitespace is a concatenation separator between two terms, else ignored
    out = []
    for k, t in enumerate(toks):
        if t[0] == "WS":
            continue
        out.append(t)
    return out


@dataclass
class _Frag:
    start: int
    end: int
    edges: list = field(default_factory=list)  # (from, symbol or None, to)


class _Builder:
    def __init__(self, n_labels: int):
        self.L = n_labels
        self.n = 0

    def state(self) -> int:
        self.n += 1
        return self.n - 1

    def symbol(self, a: int) -> _Frag:
        s, e = self.state(), self.state()
        return _Frag(s, e, [(s, a, e)])

    def concat(self, x: _Frag, y: _Frag) -> _Frag:
        return _Frag(x.start, y.end, x.edges + y.edges + [(x.end, None, y.start)])

    def alt(self, x: _Frag, y: _Frag) -> _Frag:
        s, e = self.state(), self.state()
        return _Frag(s, e, x.edges + y.edges + [(s, None, x.start), (s, None, y.start),
                                                (x.end, None, e), (y.end, None, e)])

    def star(self, x: _Frag) -> _Frag:
        s, e = self.state(), self.state()
        return _Frag(s, e, x.edges + [(s, None, x.start), (s, None, e),
                                      (x.end, None, x.start), (x.end, None, e)])

    def plus(self, x: _Frag) -> _Frag:
        s, e = self.state(), self.state()
        return _Frag(s, e, x.edges + [(s, None, x.start), (x.end, None, x.start),
                                      (x.end, None, e)])

    def opt(self, x: _Frag) -> _Frag:
        s, e = self.state(), self.state()
        return _Frag(s, e, x.edges + [(s, None, x.start), (s, None, e), (x.end, None, e)])

    def inverse(self, x: _Frag) -> _Frag:
        """R^-: reverse every edge, invert every symbol, swap start and end."""
        L = self.L

        def inv(a):
            if a is None:
                return None
            return a + L if a < L else a - L

        return _Frag(x.end, x.start, [(t, inv(a), f) for (f, a, t) in x.edges])


class _Parser:
    def __init__(self, toks, builder: _Builder):
        self.t = toks
        self.i = 0
        self.b = builder

    def peek(self):
        return self.t[self.i][0] if self.i < len(self.t) else None

    def take(self, kind):
        if self.peek() != kind:
            raise RegexError(f"expected {kind} at token {self.i}, got {self.peek()}")
        self.i += 1
        return self.t[self.i - 1]

    def alt(self):
        f = self.seq()
        while self.peek() == "|":
            self.i += 1
            f = self.b.alt(f, self.seq())
        return f

    def seq(self):
        f = self.post()
        while True:
            k = self.peek()
            if k == "CAT":
                self.i += 1
                f = self.b.concat(f, self.post())
            elif k in ("LABEL", "^", "("):
                f = self.b.concat(f, self.post())
            else:
                return f

    def post(self):
        f = self.atom()
        while self.peek() in ("*", "+", "?"):
            k = self.take(self.peek())[0]
            f = {"*": self.b.star, "+": self.b.plus, "?": self.b.opt}[k](f)
        return f

    def atom(self):
        k = self.peek()
        if k == "LABEL":
            a = self.take("LABEL")[1]
            if a >= self.b.L:
                raise RegexError(f"label {a} out of range [0, {self.b.L})")
            return self.b.symbol(a)
        if k == "^":
            self.i += 1
            return self.b.inverse(self.atom())
        if k == "(":
            self.i += 1
            f = self.alt()
            self.take(")")
            return f
        raise RegexError(f"unexpected token {k} at {self.i}")


def compile_regex(text: str, n_labels: int) -> Nfa:
    """Thompson construction followed by epsilon removal."""
    toks = _tokenize(text)
    if not toks:
        raise RegexError("empty expression")
    b = _Builder(n_labels)
    p = _Parser(toks, b)
    frag = p.alt()
    if p.i != len(toks):
        raise RegexError(f"trailing input at token {p.i}")

    n = b.n
    eps = [[] for _ in range(n)]
    sym = [[] for _ in range(n)]
    for f, a, t in frag.edges:
        (eps if a is None else sym)[f].append((a, t))

    def closure(q):
        seen = {q}
        stack = [q]
        while stack:
            x = stack.pop()
            for _, y in eps[x]:
                if y not in seen:
                    seen.add(y)
                    stack.append(y)
        return seen

    clo = [closure(q) for q in range(n)]
    trans = set()
    for q in range(n):
        for a, r in sym[q]:
            for r2 in clo[r]:
                trans.add((q, a, r2))
    starts = sorted(clo[frag.start])
    finals = [frag.end]
    return Nfa(n, n_labels, sorted(trans), starts, finals)


def inverse_nfa(nfa: Nfa) -> Nfa:
    """N^- of section 4: transitions reversed with inverted symbols, starts and
    finals swapped; it accepts R^-."""
    L = nfa.n_labels
    tr = sorted((r, a + L if a < L else a - L, q) for (q, a, r) in nfa.transitions)
    return Nfa(nfa.n_states, L, tr, list(nfa.finals), list(nfa.starts))
