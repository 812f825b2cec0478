"""The paper's operation-count model for one application of H to n_v vectors.

TEST INFRASTRUCTURE (oracle): see ``oracle/__init__.py``.

Per-stage counts and totals of Sec. 5.4 (eq. flopRealMF, eq. flopComplexMF,
eq. flopRealCM, eq. flopComplexCM), with the batch product b2 * nb2 * nb1 (and
b0 * nb0 for the cell-matrix counts) written as n_v.  That product is the number
of REAL columns: in the multilevel layout of Sec. 4.2 a complex multivector keeps
its real and imaginary parts in separate level-2 batches (b1 = c b2, level-0
batch c N_v), so for a complex operator n_v = 2 x the number of complex vectors.
n_s is the total number of projectors, E the number of cells.
"""


def _halves(n):
    return n // 2, (n + 1) // 2


def mf_real_stages(n_p, n_q, n_v, E, n_s):
    npo, _ = _halves(n_p)
    nqo, _ = _halves(n_q)
    s = n_p * n_p + n_p * n_q + n_q * n_q
    return {
        "Y0": 2 * n_v * (npo + nqo * (n_p + 1)) * s * E,
        "Y1": 6 * n_v * nqo * n_q ** 2 * (n_q + 2) * E,
        "Y2": 5 * n_v * n_q ** 3 * E,
        "Y3": 6 * n_v * n_q ** 3 * E + (3 * n_v * n_q ** 3 + 2 * n_q ** 3 + 18 * n_v * n_q ** 3) * E,
        "Y4": 6 * n_v * nqo * n_q ** 2 * (n_q + 3) * E + 2 * n_v * n_q ** 3 * E,
        "Y5": 2 * n_v * (nqo + npo * (n_q + 1)) * s * E,
        "nloc": n_v * (4 * n_p ** 3 + 1) * n_s,
    }


def mf_real_total(n_p, n_q, n_v, E, n_s):
    """eq. flopRealMF (closed form)."""
    npo, _ = _halves(n_p)
    nqo, _ = _halves(n_q)
    s = n_p * n_p + n_p * n_q + n_q * n_q
    per = (2 * n_v * (npo * (n_q + 2) + nqo * (n_p + 2)) * s
           + 6 * n_v * nqo * n_q ** 2 * (2 * n_q + 5)
           + 2 * n_q ** 3 + 34 * n_v * n_q ** 3)
    return per * E + n_v * (4 * n_p ** 3 + 1) * n_s


def mf_complex_stages(n_p, n_q, n_v, E, n_s):
    npo, _ = _halves(n_p)
    nqo, _ = _halves(n_q)
    s = n_p * n_p + n_p * n_q + n_q * n_q
    return {
        "Y0": 2 * n_v * (npo + nqo * (n_p + 1)) * s * E,
        "Y1": 6 * n_v * nqo * n_q ** 2 * (n_q + 2) * E,
        "Y2": 5 * n_v * n_q ** 3 * E,
        "Y3": 5 * n_v * n_q ** 3 * E,
        "Y4": 6 * n_v * n_q ** 3 * E + (3 * n_v * n_q ** 3 + 2 * n_q ** 3 + 18 * n_v * n_q ** 3) * E,
        "Y5": 6 * n_v * nqo * n_q ** 2 * (n_q + 3) * E + 3 * n_v * n_q ** 3 * E,
        "Y6": 2 * n_v * (nqo + npo * (n_q + 1)) * s * E,
        "nloc": n_v * (8 * n_p ** 3 + 3) * n_s,
    }


def mf_complex_total(n_p, n_q, n_v, E, n_s):
    """eq. flopComplexMF (closed form)."""
    npo, _ = _halves(n_p)
    nqo, _ = _halves(n_q)
    s = n_p * n_p + n_p * n_q + n_q * n_q
    return (2 * n_v * (npo * (n_q + 2) + nqo * (n_p + 2)) * s * E
            + 6 * n_v * nqo * n_q ** 2 * (2 * n_q + 5) * E
            + 2 * n_q ** 3 * E + 40 * n_v * n_q ** 3 * E
            + n_v * (8 * n_p ** 3 + 3) * n_s)


def cm_real_total(n_p, n_v, E, n_s):
    """eq. flopRealCM."""
    return 2 * n_v * n_p ** 6 * E + n_v * (4 * n_p ** 3 + 1) * n_s


def cm_complex_total(n_p, n_v, E, n_s):
    """eq. flopComplexCM."""
    return 6 * n_v * n_p ** 6 * E + 3 * n_v * (4 * n_p ** 3 + 1) * n_s
