"""Helpers shared by the GPU parity tests (layout conversion, oracle runs)."""
import numpy as np

import oracle as O
import paper_2603_15285_gb300 as m


def coef_to_complex(t):
    a = t.detach().cpu().double().numpy()
    return a[..., 0] + 1j * a[..., 1]


def corr_to_oracle(c_gpu_one, L):
    """Library grouped layout [nc][2][2] -> the oracle's full c^l_mn array."""
    a = m.corr_pairs(c_gpu_one.detach().cpu().double().numpy())
    z = a[..., 0] + 1j * a[..., 1]          # [nc][2]
    out = np.zeros(O.c_size(L), complex)
    for e, (mm, nn, l) in enumerate(m.corr_layout(L)):
        if nn > mm:                          # empty partner slot
            assert z[e, 0] == 0 and z[e, 1] == 0
            continue
        out[O.c_index(l, mm, nn)] = z[e, 0]
        out[O.c_index(l, nn, mm)] = z[e, 1]
    # negative images: c_{-m,-n} = (-1)^{m+n} conj(c_mn)
    for l in range(L + 1):
        for mm in range(-l, l + 1):
            for nn in range(-l, l + 1):
                i = O.c_index(l, mm, nn)
                if out[i] == 0:
                    out[i] = (-1) ** (mm + nn) * np.conj(out[O.c_index(l, -mm, -nn)])
    return out


def oracle_align(w, parts, temps, **kw):
    return O.align_batch(parts, temps, S=w.n_shells, r_max=w.r_max, L0=w.L0, K=w.K, P=w.P,
                         M_iter=w.M_iter, L_sched=w.L_sched, **kw)
