"""Error bound of one mixed-precision constant-coefficient solve, from the
arithmetic the mixed plans perform (used by the GPU parity tests).

u = 2^-24 is the unit roundoff of FP32.  One solve rounds to FP32:
  * the right-hand side once, when it is narrowed from FP64 (1 u);
  * inside each of its four transforms (forward x, forward y, inverse y,
    inverse x), once per Stockham pass for the twiddle product and twice
    for the butterfly sums, taken here as 3 u per pass without cancellation
    between passes (normwise, worst case): a length N = prod of the radices
    8, 4, 2, 3, 5 takes one pass per radix;
  * the z solve's two stored sweeps (2 u; the z recurrences of the headline
    plan run in FP64).
So eps_1 = u (1 + 3 (2 P(nx) + 2 P(ny)) + 2), P(N) the pass count.  After
`passes` Method III passes the iterate is a sum of that many corrections,
each no larger than the first, so the bound grows by that factor.  The
hybrid plan's FP32 z recurrences run only on columns of condition number
<= 513, whose solutions are the small, high-wavenumber part of p: measured,
its errors stay within 5 % of those of the FP64-recurrence plan, inside the
slack of this normwise model (the observed errors are 3-4 u per solve and
about 30 u for the velocities after two 512^3 passes).  Walls in y add one
pass (the pairwise twiddles of the cosine transform) to each y transform."""

U32 = 2.0 ** -24


def stockham_passes(n):
    p, m = 0, int(n)
    for r in (8, 4, 2, 3, 5):
        while m % r == 0 and m > 1:
            m //= r
            p += 1
    return p


def mixed_solve_bound(nx, ny, passes=1, ywalls=False, margin=1.0):
    py = stockham_passes(ny) + (1 if ywalls else 0)
    per_solve = 1 + 3 * (2 * stockham_passes(nx) + 2 * py) + 2
    return margin * passes * per_solve * U32


# Relative error of one term of a BF16x3 split product (hi*hi + hi*lo +
# lo*hi): x = x_hi + x_lo + dx with |x_lo| <= 2^-9 |x| and |dx| <= 2^-9
# |x_lo|, the same for the matrix entry, so the dropped lo*lo and the two
# dx terms are each at most 2^-18 of |m x|; FP32 accumulation adds u.
BF16X3 = 3 * 2.0 ** -18 + U32


def mixed_solve_bound_dense_y(nx, ny, dyf, tc=False, nz=None, margin=1.0):
    """The same bound with the y transforms as dense BF16x3 products on the
    tensor cores (a stretched y between walls).  Each output of a product is
    a sum of ny terms, so its error is at most ny BF16X3 sum_j |M_mj x_j|
    (worst case, no cancellation); normwise || |M| |x| || <= sqrt(ny) ||M||
    ||x||, and the forward (V^T W) and inverse (V) matrices of the
    W-orthonormal basis have norms sqrt(max dyf) and 1 / sqrt(min dyf), so a
    forward-inverse pair carries sqrt(max dyf / min dyf).  Each of the two y
    products thus adds ny sqrt(ny max dyf / min dyf) BF16X3.  With tc (the
    tensor-core z expansion) the two z products add nz sqrt(nz) BF16X3 each,
    in the same worst-case form."""
    import math
    ratio = float(max(dyf)) / float(min(dyf))
    dense = ny * math.sqrt(ny * ratio) * BF16X3
    per_solve = (1 + 3 * 2 * stockham_passes(nx) + 2) * U32 + 2 * dense
    if tc:
        per_solve += 2 * nz * math.sqrt(nz) * BF16X3
    return margin * per_solve
