"""NumPy emulation of the packed-FP16 gather kernel's arithmetic (gather_split = 4), in its
order, for the rounding-point test (test infrastructure; it shares nothing with the CUDA code
but this description of what the kernel computes).

For output pixel q and tap t = (ty, tx) of a 33 x 33 grid, the gather of Eq. 5 sums
G[q, t] x[q - o(t)], o(t) = (ty - 16, tx - 16), x zero outside the frame.  The kernel rounds
beta and H to the operand type, forms G = beta H in FP32 and rounds it to FP16, stages x in
FP16 and accumulates:

- The four groups of warps take tap columns [8 g, 8 g + 8); output rows pair up as (r, r + 1)
  with r even, and row r + 1 takes tap rows one further than row r ("parity" 1).
- Main chunks c = 0 .. 10, pairs p = 3 c + j (j < 3), tap columns in order: tap row p - 1 + parity
  (skipped outside 0 .. 32).  Each product goes into one of two FP16 sums, by the parity of its
  tap column (one rounding per FMA); the sums start at 0 in every chunk and are added into the
  FP32 sum at the chunk's end, the even one first.
- The last chunk: tap row 32 of the group's tap columns for parity 0 only, into fresh FP16 sums;
  then tap column 32, tap rows [9 g, min(9 g + 9, 33)), straight into the FP32 sum (one rounding
  per product); then the FP16 sums are added, the even one first.
- y = ((s_0 + s_1) + s_2) + s_3 in FP32.
"""
import numpy as np

TAPS = 33
HALF = TAPS // 2


def _shifted(x16, ty, tx):
    """x[q - o(t)] for all q, zero outside the frame (float64 array of FP16 values)."""
    h, w = x16.shape[:2]
    dy, dx = ty - HALF, tx - HALF
    out = np.zeros_like(x16)
    ys, ye = max(0, dy), min(h, h + dy)
    xs, xe = max(0, dx), min(w, w + dx)
    if ys < ye and xs < xe:
        out[ys:ye, xs:xe] = x16[ys - dy : ye - dy, xs - dx : xe - dx]
    return out


def _f16(v):
    return v.astype(np.float16).astype(np.float64)


def _f32(v):
    return v.astype(np.float32).astype(np.float64)


def gather_h2(x, beta, Hb, operand_round):
    """x [h, w, C], beta [h, w, K], Hb [K, 33 * 33]; operand_round rounds beta and H to the
    MMA's operand type (FP16 or BF16, as float64 values)."""
    h, w, C = x.shape
    G = operand_round(beta.reshape(h * w, -1).astype(np.float64)) @ operand_round(Hb.astype(np.float64))
    G16 = _f16(G).reshape(h, w, TAPS, TAPS)
    x16 = _f16(np.asarray(x, dtype=np.float64))
    xs = {}

    def xat(ty, tx):
        if (ty, tx) not in xs:
            xs[(ty, tx)] = _shifted(x16, ty, tx)
        return xs[(ty, tx)]

    y = {}
    for parity in (0, 1):
        sums = []
        for g in range(4):
            s32 = np.zeros((h, w, C))
            for c in range(11):
                s16 = [np.zeros((h, w, C)), np.zeros((h, w, C))]
                for j in range(3):
                    ty = 3 * c + j - 1 + parity
                    if not 0 <= ty < TAPS:
                        continue
                    for u in range(8):
                        tx = 8 * g + u
                        s16[u & 1] = _f16(G16[:, :, ty, tx][:, :, None] * xat(ty, tx) + s16[u & 1])
                s32 = _f32(_f32(s32 + s16[0]) + s16[1])
            s16 = [np.zeros((h, w, C)), np.zeros((h, w, C))]
            if parity == 0:
                for u in range(8):
                    tx = 8 * g + u
                    s16[u & 1] = _f16(G16[:, :, TAPS - 1, tx][:, :, None] * xat(TAPS - 1, tx) + s16[u & 1])
            for ty in range(9 * g, min(9 * g + 9, TAPS)):
                s32 = _f32(s32 + G16[:, :, ty, TAPS - 1][:, :, None] * xat(ty, TAPS - 1))
            s32 = _f32(_f32(s32 + s16[0]) + s16[1])
            sums.append(s32)
        y[parity] = _f32(_f32(_f32(sums[0] + sums[1]) + sums[2]) + sums[3])
    rows = (np.arange(h) % 2)[:, None, None]
    return np.where(rows == 0, y[0], y[1])
