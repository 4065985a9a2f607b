#!/usr/bin/env python3
"""Generates ring_network.inc: the paired multiply-accumulate networks of the staged ring kernel.

For a ring R_{2,N} the generated device function ring_mac_pairs_n<N>(acc, d, r) adds r * d to the
N ring accumulators, r an N-bit mask (phi_S of a field coefficient, paper Sec. 2.2) and d the W
packets of an embedded source block (W = N - 1 for the all-one polynomials, 6 for N = 9; its
coefficients at x^W and above are zero, phi_E, Sec. 2.3.2 and Sec. 2.4.2). Multiplying by x^s rotates the packets by s (Sec. 3), so r * d is the XOR of one
rotation per set bit of r.

The set bits are consumed in increasing order and fused two at a time: for consecutive set bits
(s1, s2) every accumulator t receives d[t - s1] ^ d[t - s2] in one three-input XOR, instead of
two separate passes; a leftover bit is a plain rotation. The walk over bit positions is a
finite automaton whose state is (pending set bit or none, position); each state is one labelled
block that tests one bit of the warp-uniform r and branches forward to a static target, so no
register is ever indexed at run time and no jump table is used.

Run from this directory: python gen_ring_network.py  (rewrites ring_network.inc).
"""
import os

RINGS = (3, 5, 9, 11, 13)


def ring_w(N):
    """Field degree carried by R_{2,N}: N - 1 for the all-one polynomials, 6 for N = 9 (the ESP
    x^6 + x^3 + 1); the source's packets at index >= w are the embedding's zeros."""
    return 6 if N == 9 else N - 1


def emit_ring(N):
    out = []
    out.append("// R_{2,%d}: %d labelled states, %d fused pairs." % (N, (N + 1) + N * (N + 1) // 2, N * (N - 1) // 2))
    out.append("template <int WORDS>")
    out.append("__device__ __forceinline__ void ring_mac_pairs_n%d(uint32_t (&acc)[%d][WORDS], "
               "const uint32_t (&d)[%d][WORDS], const uint32_t r) {" % (N, N, ring_w(N)))
    # X_s: no pending bit, about to test position s.  P_p_s: bit p pending, about to test s.
    for s in range(N):
        if s:
            out.append("X_%d:" % s)
        nxt_set = "P_%d_%d" % (s, s + 1)
        out.append("  if (r & (1u << %d)) goto %s;" % (s, nxt_set))
        if s + 1 < N:
            out.append("  goto X_%d;" % (s + 1))
        else:
            out.append("  goto DONE;")
    for p in range(N):
        for s in range(p + 1, N + 1):
            out.append("P_%d_%d:" % (p, s))
            if s == N:
                out.append("  xor_rotated<%d, WORDS, %d>(acc, d);" % (N, p))
                out.append("  goto DONE;")
                continue
            after = "X_%d" % (s + 1) if s + 1 < N else "DONE"
            out.append("  if (r & (1u << %d)) {" % s)
            out.append("    xor_pair<%d, WORDS, %d, %d>(acc, d);" % (N, p, s))
            out.append("    goto %s;" % after)
            out.append("  }")
            out.append("  goto P_%d_%d;" % (p, s + 1))
    out.append("DONE:")
    out.append("  return;")
    out.append("}")
    return "\n".join(out)


def source():
    """The text of ring_network.inc."""
    body = ["// Generated by gen_ring_network.py -- do not edit by hand.",
            "// Paired ring multiply-accumulate automata (see the generator's docstring)."]
    for N in RINGS:
        body.append(emit_ring(N))
    body.append("")
    body.append("template <int N, int WORDS>")
    body.append("__device__ __forceinline__ void ring_mac_pairs(uint32_t (&acc)[N][WORDS], "
                "const uint32_t (&d)[RingDim<N>::W][WORDS], const uint32_t r) {")
    for N in RINGS:
        body.append("  if constexpr (N == %d) ring_mac_pairs_n%d<WORDS>(acc, d, r);" % (N, N))
    body.append("}")
    return "\n".join(body) + "\n"


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "ring_network.inc"), "w") as f:
        f.write(source())


if __name__ == "__main__":
    main()
