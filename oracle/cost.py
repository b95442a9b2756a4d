"""Operation counts and the throughput metric (test infrastructure only).

* Sec. III.F, Eq. (13): template method per block, z_basic = N T (5 log2 N + 6).
* Eq. (14): folded first stage, z_first = N T (5/w log2(N/w) + 6 + 2/w).
* Eq. (15): z_total = z_first + 4 p w f(w, rho_I) T + N p (5 log2 N + 6),
  with f(w, rho_I) the first-stage candidates per template and block.
* Sec. IV.B.2: throughput = (seconds of data) x (templates) / (wall seconds),
  the number of templates filtered in real time.

Pinned by the worked example of Sec. IV.B.2 / Table II (64 s against 6250
templates in ~100 ms is 4.0e6), stored in tests/golden/throughput_table2.json.
"""
from __future__ import annotations

import math


def z_basic(n, t):
    return n * t * (5.0 * math.log2(n) + 6.0)


def z_first(n, t, w):
    return n * t * (5.0 / w * math.log2(n / w) + 6.0 + 2.0 / w)


def z_total(n, t, w, p, f_trig):
    return z_first(n, t, w) + 4.0 * p * w * f_trig * t + n * p * (5.0 * math.log2(n) + 6.0)


def throughput(seconds, templates, wall_seconds):
    return seconds * templates / wall_seconds
