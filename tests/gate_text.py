"""Text form of qs_gate arrays for the host-side C++ checks under tests/cpp:
one gate per line, `kind nw w0 w1 w2 p0 p1 p2 [param_idx] has_dense [8 doubles]`
(param_idx only when `pidx` is true)."""


def gate_lines(qs, gates, pidx=False):
    cg = qs.CGates(gates)
    out = []
    for i in range(cg.n):
        g = cg.arr[i]
        row = [g.kind, g.nw, g.w[0], g.w[1], g.w[2], repr(g.p[0]), repr(g.p[1]), repr(g.p[2])]
        if pidx:
            row.append(g.param_idx)
        if g.dense:
            row += [1] + [repr(g.dense[e]) for e in range(8)]
        else:
            row += [0]
        out.append(" ".join(str(x) for x in row))
    return out
