"""Instruction-throughput roofline of Sec. 4 (Eq. 6-11, Eq. 20).

Reporting arithmetic for the benchmark; nothing here runs on the search path.

  attainable(pi, beta, gamma, I_mem, I_cop) = min(pi, beta*I_mem, gamma*I_cop)  (Eq. 6)
  I_mem of a level-3 distance kernel that writes the M x N matrix ~ D/2         (Eq. 7)
  COP budget per score  C <= 2 D gamma / pi                                    (Eq. 8-9)
  PartialReduce intensities: I_cop = 2D / C                                    (Eq. 11)
  I_mem = 2MND / (4 (MD + MND/ib + 2ML))                                       (Eq. 20)
Units: pi in FLOP/s, beta in bytes/s, gamma in COP/s.

GB300's gamma is derived from unit counts and the clock: 152 SMs, each
issuing per clock 64 lanes of ALU-pipe work (integer, logic, compare,
min/max, select) and 128 lanes of FMA-pipe work (FP32 add/mul/fma), at
2.07 GHz. PartialReduce's compares and selects are ALU-pipe COPs.
"""

GB300_SMS = 152
GB300_ALU_LANES_PER_SM = 64
GB300_FMA_LANES_PER_SM = 128
GB300_MAX_CLOCK_HZ = 2.07e9


def attainable(pi, beta, gamma, i_mem, i_cop):
    """Eq. 6: the attainable FLOP/s of a kernel under the three roofs."""
    return min(pi, beta * i_mem, gamma * i_cop)


def binding_roof(pi, beta, gamma, i_mem, i_cop):
    roofs = {"tensor": pi, "hbm": beta * i_mem, "cop": gamma * i_cop}
    return min(roofs, key=roofs.get)


def i_mem_dense_scores(M, N, D, bytes_per_score=4):
    """Eq. 7: FLOP per byte when the M x N score matrix is written out."""
    return 2.0 * M * N * D / (bytes_per_score * M * N)


def cop_budget(D, gamma, pi):
    """Eq. 9: the most COPs per score that keep a kernel off the COP roof."""
    return 2.0 * D * gamma / pi


def i_cop(D, C):
    """Eq. 11: FLOP per COP of PartialReduce with C COPs per score."""
    return 2.0 * D / C


def i_mem_partial_reduce(M, N, D, L, ib, elem_bytes=4):
    """Eq. 20: FLOP per byte of the blocked PartialReduce (query block ib)."""
    b = elem_bytes
    return 2.0 * M * N * D / (b * M * D + b * M * N * D / ib + 2 * 4 * M * L)


def gb300_gamma(pipe="alu", sms=GB300_SMS, clock_hz=GB300_MAX_CLOCK_HZ):
    """Peak COP/s of one GB300 on the ALU or FMA pipe (lanes x SMs x clock)."""
    lanes = GB300_ALU_LANES_PER_SM if pipe == "alu" else GB300_FMA_LANES_PER_SM
    return float(sms * lanes * clock_hz)


def report(M, N, D, seconds, pi, beta, gamma, C, bytes_moved):
    """Eq. 6 for one measured launch: the three roofs, the binding one, and
    the measured FLOP/s against the attainable bound. C = COPs per score on
    the pipe gamma counts; bytes_moved = DRAM bytes of the launch."""
    flops = 2.0 * M * N * D
    i_mem = flops / bytes_moved
    ic = i_cop(D, C) if C > 0 else float("inf")
    roofs = {"tensor": pi, "hbm": beta * i_mem, "cop": gamma * ic}
    bound = min(roofs, key=roofs.get)
    measured = flops / seconds
    return {"flops": flops, "I_MEM": i_mem, "I_COP": ic, "C": C, "roofs": roofs,
            "binding": bound, "attainable": roofs[bound], "measured": measured,
            "fraction_of_attainable": measured / roofs[bound]}
