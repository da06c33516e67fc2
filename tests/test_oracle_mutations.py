"""Planted mistakes in a copy of the oracle fail its pins (CPU).

Each case copies oracle/ with one source line changed, plus tests/ and synth/,
into a temporary directory and runs there the pin module for that part of the
oracle; the module must fail, on an assertion (not on a build error).  The
cases run side by side, one subprocess each.  This is
what ties the pins to something other than the oracle itself: a plausible
slip in an operation, an index, an order, a sign or a bound breaks at least
one of them.  The mistakes are planted in the oracle only, on the CPU.
"""

import os
import shutil
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CORE = "test_oracle_pins.py"
CONF = "test_oracle_conf_pins.py"
SWAP = "test_oracle_swap_pins.py"
COLOUR = "test_oracle_colour_pins.py"
COMB = "test_oracle_combined_pins.py"
TRACK = "test_oracle_track_pins.py"
MESH = "test_oracle_mesh_pins.py"
SHARD = "test_oracle_shard_pins.py"

# (pin module, mistake, original text, planted text)
MUTANTS = [
    # allocation, integration, raycast (Sec. 3-4)
    (CORE, "voxel centre instead of corner", "                    float px = (float)(bx * 8 + lx) * vs;",
     "                    float px = ((float)(bx * 8 + lx) + 0.5f) * vs;"),
    (CORE, "no truncation of f", "                    if (f > 1.0f) f = 1.0f;", ""),
    (CORE, "sign of eta", "                    float eta = d - Z;", "                    float eta = Z - d;"),
    (CORE, "pose inverse not transposed", "        for (int j = 0; j < 3; ++j) M[4 * i + j] = (float)R[j][i];",
     "        for (int j = 0; j < 3; ++j) M[4 * i + j] = (float)R[i][j];"),
    (CORE, "DDA drops the last block", "    while (left[0] + left[1] + left[2] > 0) {",
     "    while (left[0] + left[1] + left[2] > 1) {"),
    (CORE, "wrong excess index", "        if (e->offset < 1) return -1;\n        idx = s->nb + e->offset - 1;",
     "        if (e->offset < 1) return -1;\n        idx = s->nb + e->offset;"),
    (CORE, "wrong hash prime", "    uint32_t hx = (uint32_t)x * 73856093u;", "    uint32_t hx = (uint32_t)x * 73856092u;"),
    (CORE, "pixel index without rounding", "                    int pix = (int)(u + 0.5f) + (int)(v + 0.5f) * W;",
     "                    int pix = (int)(u) + (int)(v) * W;"),
    (CORE, "depth by a reciprocal multiply", "    for (long long i = 0; i < n; ++i) out[i] = (float)raw[i] / 1000.0f;",
     "    for (long long i = 0; i < n; ++i) out[i] = (float)raw[i] * 0.001f;"),
    (CORE, "refinement step sign", "                t = t + F * tmu;\n            }\n            float p[3];",
     "                t = t - F * tmu;\n            }\n            float p[3];"),
    (CORE, "normal sign", "                float fm = trilinear(s, qm, &obs);\n                g[a] = fp - fm;",
     "                float fm = trilinear(s, qm, &obs);\n                g[a] = fm - fp;"),
    (CORE, "no weight cap", "                    Wt[i] = den < max_w ? den : max_w;", "                    Wt[i] = den;"),
    (CORE, "capped weight as the divisor", "                    F[i] = num / den;",
     "                    F[i] = num / (den < max_w ? den : max_w);"),
    (CORE, "behind-surface skip dropped", "                    if (eta < -mu) continue;", ""),
    (CORE, "f not divided by mu", "                    float f = eta / mu;", "                    float f = eta;"),
    (CORE, "no one-pixel image border", "    const float umax = (float)(W - 2), vmax = (float)(H - 2);",
     "    const float umax = (float)(W - 1), vmax = (float)(H - 1);"),
    (CORE, "segment ends at the surface", "    float z1 = d + mu;", "    float z1 = d;"),
    (CORE, "segment starts at the surface", "    float z0 = d - mu;", "    float z0 = d;"),
    (CORE, "near end not clamped in front of the camera", "    if (z0 < 1e-3f) z0 = 1e-3f;", ""),
    (CORE, "depth range ignored in allocation", "    if (d < s->z_min || d > s->z_max) return 0;", ""),
    (CORE, "pose inverse translation sign", "        for (int j = 0; j < 3; ++j) acc -= R[j][i] * t[j];",
     "        for (int j = 0; j < 3; ++j) acc += R[j][i] * t[j];"),
    (CORE, "voxels behind the camera not skipped", "                    if (Z <= 0.0f) continue;\n                    float u",
     "                    float u"),
    (CORE, "raycast starts at 0, not z_min", "            float t = s->z_min;", "            float t = 0.0f;"),
    (CORE, "normal where a sampled voxel is unobserved",
     "                float fm = trilinear(s, qm, &obs);\n                g[a] = fp - fm;\n            }\n            float gl = sqrtf((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);\n            if (obs && gl > 0.0f) {",
     "                float fm = trilinear(s, qm, &obs);\n                g[a] = fp - fm;\n            }\n            float gl = sqrtf((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);\n            if (gl > 0.0f) {"),
    (CORE, "no minimum raycast step",
     "                if (step < ts) step = ts;\n                t = t + step;\n            }\n"
     "            if (state != BEHIND_SURFACE) continue;\n            for (int r = 0; r < 2; ++r) {\n"
     "                for (int i = 0; i < 3; ++i) q[i]",
     "                t = t + step;\n            }\n"
     "            if (state != BEHIND_SURFACE) continue;\n            for (int r = 0; r < 2; ++r) {\n"
     "                for (int i = 0; i < 3; ++i) q[i]"),
    (CORE, "trilinear x weights reversed", "    float c00 = lerpf(c000, c100, fr[0]);",
     "    float c00 = lerpf(c100, c000, fr[0]);"),
    (CORE, "trilinear z weights reversed", "    return lerpf(c0, c1, fr[2]);\n}\n\nenum",
     "    return lerpf(c1, c0, fr[2]);\n}\n\nenum"),
    (CORE, "trilinear y weights reversed", "\n    float c0 = lerpf(c00, c10, fr[1]);",
     "\n    float c0 = lerpf(c10, c00, fr[1]);"),
    (CORE, "trilinear corners y and z swapped", "    float c010 = voxel_value(s, x, y + 1, z, &o[2])",
     "    float c010 = voxel_value(s, x, y, z + 1, &o[2])"),
    (CORE, "sdf starts at 0", "        s->sdf[(size_t)ptr * ORC_BLOCK3 + i] = 1.0f;",
     "        s->sdf[(size_t)ptr * ORC_BLOCK3 + i] = 0.0f;"),
    (CORE, "coarse search without the step back",
     "                        t = t - tB;\n                        state = SEARCH_BLOCK_FINE;\n                    }\n"
     "                    continue;\n                }\n                if (!alloc) {\n"
     "                    if (state == SEARCH_BLOCK_FINE) t = t + tmu;\n                    else state = SEARCH_BLOCK_COARSE;\n"
     "                    continue;\n                }\n                int obs",
     "                        state = SEARCH_BLOCK_FINE;\n                    }\n"
     "                    continue;\n                }\n                if (!alloc) {\n"
     "                    if (state == SEARCH_BLOCK_FINE) t = t + tmu;\n                    else state = SEARCH_BLOCK_COARSE;\n"
     "                    continue;\n                }\n                int obs"),
    # learned confidence weight
    (CONF, "bf16 by truncation", "    u += 0x7fffu + lsb;\n    u &= 0xffff0000u;", "    u &= 0xffff0000u;"),
    (CONF, "bf16 ties away from zero", "    u += 0x7fffu + lsb;", "    u += 0x8000u; (void)lsb;"),
    (CONF, "feature clamp at 3", "                if (f > 4.0) f = 4.0;\n                if (f < -4.0) f = -4.0;",
     "                if (f > 3.0) f = 3.0;\n                if (f < -3.0) f = -3.0;"),
    (CONF, "patch index transposed", "            x[(i + 3) * 7 + (j + 3)] = f;", "            x[(j + 3) * 7 + (i + 3)] = f;"),
    (CONF, "feature sign", "                f = (d - dc) / (double)mu;", "                f = (dc - d) / (double)mu;"),
    (CONF, "normal cross product order",
     "        double n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};",
     "        double n[3] = {b[1] * a[2] - b[2] * a[1], b[2] * a[0] - b[0] * a[2], b[0] * a[1] - b[1] * a[0]};"),
    (CONF, "W1 read with the wrong stride",
     "        for (int k = 0; k < ORC_NF; ++k) acc += maybe_bf16(W1[m * ORC_NF + k], round_bf16) * xin[k];",
     "        for (int k = 0; k < ORC_NF; ++k) acc += maybe_bf16(W1[k * ORC_NH + m], round_bf16) * xin[k];"),
    (CONF, "b1 dropped", "        a1[m] = relu(acc + b1[m]);", "        a1[m] = relu(acc);"),
    (CONF, "features not rounded to bfloat16",
     "    for (int k = 0; k < ORC_NF; ++k) xin[k] = maybe_bf16(x[k], round_bf16);",
     "    for (int k = 0; k < ORC_NF; ++k) xin[k] = x[k];"),
    (CONF, "layer-2 input not rounded to bfloat16", "        a1in[m] = maybe_bf16(a1[m], round_bf16);",
     "        a1in[m] = a1[m];"),
    (CONF, "no ReLU on layer 2", "        a2[n] = relu(acc + b2[n]);", "        a2[n] = acc + b2[n];"),
    (CONF, "b2 dropped", "        a2[n] = relu(acc + b2[n]);", "        a2[n] = relu(acc);"),
    (CONF, "b3 dropped", "    double o = b3[0];", "    double o = 0.0; (void)b3;"),
    (CONF, "gradient not averaged", "        double dout = (p - t) / n;", "        double dout = (p - t);"),
    (CONF, "layer-2 gradient not masked", "            d2[k] = h2[k] > 0.0 ? dout * w3[k] : 0.0;",
     "            d2[k] = dout * w3[k];"),
    (CONF, "layer-1 gradient not masked", "            d1[m] = h1[m] > 0.0 ? acc : 0.0;", "            d1[m] = acc;"),
    (CONF, "W2 gradient transposed",
     "            for (int m = 0; m < ORC_NH; ++m) gW2[a * ORC_NH + m] += d2[a] * maybe_bf16(h1[m], round_bf16);",
     "            for (int m = 0; m < ORC_NH; ++m) gW2[m * ORC_NH + a] += d2[a] * maybe_bf16(h1[m], round_bf16);"),
    (CONF, "sign of the label term", "        loss += (o > 0 ? o : 0.0) - o * t + log1p(exp(-fabs(o)));",
     "        loss += (o > 0 ? o : 0.0) + o * t + log1p(exp(-fabs(o)));"),
    # swapping (Sec. 5)
    (SWAP, "fusion weights crossed", "    float num = *W * *F + Wh * Fh;", "    float num = Wh * *F + *W * Fh;"),
    (SWAP, "host value replaces the fused one", "    *F = num / den;\n    *W = den < max_w",
     "    *F = Fh; (void)num;\n    *W = den < max_w"),
    (SWAP, "a block waiting for its host data swapped out",
     "    return e->ptr >= 0 && s->swap_state[idx] == ORC_SW_DEVICE && s->frame - s->touch[idx] >= s->swap_idle;",
     "    return e->ptr >= 0 && s->frame - s->touch[idx] >= s->swap_idle;"),
    (SWAP, "no weight clamp", "    *W = den < max_w ? den : max_w;", "    *W = den;"),
    (SWAP, "host weight 0 not skipped", "    if (!(Wh > 0.0f)) return;\n    if (!(*W > 0.0f)) {",
     "    if (!(*W > 0.0f) && (Wh > 0.0f)) {"),
    (SWAP, "device weight 0 not taken over", "    if (!(*W > 0.0f)) {\n        *F = Fh;", "    if (0) {\n        *F = Fh;"),
    (SWAP, "descending key in a chain",
     "packed_key(&s->entries[chain[j - 1]]) > packed_key(&s->entries[idx])",
     "packed_key(&s->entries[chain[j - 1]]) < packed_key(&s->entries[idx])"),
    (SWAP, "buckets in reverse order",
     "for (int h = 0; h < s->nb && n < cap; ++h) {\n        if (s->entries[h].ptr < -1) continue;",
     "for (int hh = 0; hh < s->nb && n < cap; ++hh) {\n        const int h = s->nb - 1 - hh;\n"
     "        if (s->entries[h].ptr < -1) continue;"),
    (SWAP, "freed block not returned",
     "        s->block_free[s->block_top++] = ptr;\n    }\n    free(sel);\n    s->swapped_out += n;",
     "    }\n    free(sel);\n    s->swapped_out += n;"),
    (SWAP, "swapped-out key inserted again", "        if (e->x == bx && e->y == by && e->z == bz) { /* present */",
     "        if (e->x == bx && e->y == by && e->z == bz && e->ptr != -1) { /* present */"),
    (SWAP, "blocks met again not stamped", "            touch_entry(s, e);\n            return;\n        }",
     "            return;\n        }"),
    (SWAP, "allocation count not advanced", "    if (s->swap_on) ++s->frame;", ""),
    (SWAP, "fused entry left waiting",
     "        s->swap_state[idx] = ORC_SW_DEVICE;\n    }\n    free(sel);\n    s->swapped_in += n;",
     "    }\n    free(sel);\n    s->swapped_in += n;"),
    (SWAP, "swap-in ignores the bound", "    const int n = select_entries(s, wants_in, sel, s->swap_k);",
     "    free(sel);\n    sel = (int32_t *)malloc(sizeof(int32_t) * (size_t)(s->nb + s->ne));\n"
     "    const int n = select_entries(s, wants_in, sel, s->nb + s->ne);"),
    (SWAP, "idle test off by one", "s->frame - s->touch[idx] >= s->swap_idle", "s->frame - s->touch[idx] > s->swap_idle"),
    # colour voxels (Sec. 3.1)
    (COLOUR, "colour outside the band", "                    if (cf && eta <= mu) colour_update",
     "                    if (cf) colour_update"),
    (COLOUR, "band of 2 mu", "                    if (cf && eta <= mu) colour_update",
     "                    if (cf && eta <= 2.0f * mu) colour_update"),
    (COLOUR, "rounding by truncation", "        int q = (int)(nc + 0.5f);", "        int q = (int)(nc);"),
    (COLOUR, "colour weight not capped", "    c[3] = (uint8_t)(nw < (float)s->max_w ? nw : (float)s->max_w);",
     "    c[3] = (uint8_t)nw;"),
    (COLOUR, "bilinear axes swapped", "    float a = uc - (float)u0, b = vc - (float)v0;",
     "    float b = uc - (float)u0, a = vc - (float)v0;"),
    (COLOUR, "extrinsic ignored", "    float Xc = row_apply(&cf->T[0], X, Y, Z);", "    float Xc = X; (void)row_apply;"),
    (COLOUR, "channels reversed", "        float p00 = (float)P[((size_t)v0 * cf->Wc + u0) * 3 + ch];",
     "        float p00 = (float)P[((size_t)v0 * cf->Wc + u0) * 3 + (2 - ch)];"),
    (COLOUR, "unweighted colour mean", "        float nc = (wc * (float)c[ch] + obs) / (wc + 1.0f);",
     "        float nc = ((float)c[ch] + obs) / 2.0f;"),
    (COLOUR, "colour weight steps by 2", "    float nw = wc + 1.0f;", "    float nw = wc + 2.0f;"),
    (COLOUR, "point colour with y and z strides swapped",
     "        memcpy(o, &s->rgbw[((size_t)ptr * ORC_BLOCK3 + (g[0] & 7) + 8 * (g[1] & 7) + 64 * (g[2] & 7)) * 4], 4);",
     "        memcpy(o, &s->rgbw[((size_t)ptr * ORC_BLOCK3 + (g[0] & 7) + 64 * (g[1] & 7) + 8 * (g[2] & 7)) * 4], 4);"),
    (COLOUR, "point colour from floor(q)", "            else g[a] = (int)floorf(q + 0.5f);",
     "            else g[a] = (int)floorf(q);"),    # combined map (Sec. 7.2), depth tracker (Sec. 4.1.1), Marching Cubes (Sec. 4)
    (COMB, "combined sum not normalised", "    return dsum > 0.0f ? num / dsum : 1.0f;", "    return dsum > 0.0f ? num : 1.0f;"),
    (COMB, "sign of a combined term", "        num = num + Wt * F;", "        num = num - Wt * F;"),
    (COMB, "weight taken at one corner", "    *Wt = out[1];", "    *Wt = w[0];"),
    (COMB, "submap pose transposed", "        q[r] = row_apply(P + 4 * r, X[0], X[1], X[2]) * inv_s;",
     "        q[r] = (((P[r] * X[0] + P[4 + r] * X[1]) + P[8 + r] * X[2]) + P[4 * r + 3]) * inv_s;"),
    (COMB, "first submap only",
     "    for (int i = 0; i < n; ++i) {\n        float q[3];\n        if (!submap_coords(P + 16 * i, X, inv_s, q)) continue;\n        float F, Wt;",
     "    for (int i = 0; i < 1 && i < n; ++i) {\n        float q[3];\n        if (!submap_coords(P + 16 * i, X, inv_s, q)) continue;\n        float F, Wt;"),
    (COMB, "allocation test on the first submap only",
     "    for (int i = 0; i < n; ++i) {\n        float q[3];\n        if (!submap_coords(P + 16 * i, X, inv_s, q)) continue;\n        int bx",
     "    for (int i = 0; i < 1 && i < n; ++i) {\n        float q[3];\n        if (!submap_coords(P + 16 * i, X, inv_s, q)) continue;\n        int bx"),
    (COMB, "corner bits y and z swapped",
     "        int gx = x + (k & 1), gy = y + ((k >> 1) & 1), gz = z + ((k >> 2) & 1);",
     "        int gx = x + (k & 1), gy = y + ((k >> 2) & 1), gz = z + ((k >> 1) & 1);"),
    (COMB, "x weights reversed", "        float c00 = lerpf(v[m][0], v[m][1], fr[0]);",
     "        float c00 = lerpf(v[m][1], v[m][0], fr[0]);"),
    (COMB, "unallocated voxel value 0", "            c[k] = 1.0f;\n            w[k] = 0.0f;",
     "            c[k] = 0.0f;\n            w[k] = 0.0f;"),
    (COMB, "default 0 where unobserved", "    return dsum > 0.0f ? num / dsum : 1.0f;", "    return dsum > 0.0f ? num / dsum : 0.0f;"),
    (TRACK, "cross product order in the Jacobian",
     "            const float J[6] = {pw[1] * Np[2] - pw[2] * Np[1], pw[2] * Np[0] - pw[0] * Np[2],\n"
     "                                pw[0] * Np[1] - pw[1] * Np[0], Np[0], Np[1], Np[2]};",
     "            const float J[6] = {Np[1] * pw[2] - Np[2] * pw[1], Np[2] * pw[0] - Np[0] * pw[2],\n"
     "                                Np[0] * pw[1] - Np[1] * pw[0], Np[0], Np[1], Np[2]};"),
    (TRACK, "update multiplied on the right", "            for (int m = 0; m < 3; ++m) acc += R[i][m] * (double)T[4 * m + j];",
     "            for (int m = 0; m < 3; ++m) acc += (double)T[4 * i + m] * R[m][j];"),
    (TRACK, "association without rounding",
     "            const size_t o = 4 * ((size_t)(int)(vr + 0.5f) * Wr + (int)(ur + 0.5f));",
     "            const size_t o = 4 * ((size_t)(int)(vr) * Wr + (int)(ur));"),
    (TRACK, "association through the live pose", "    float M[16];\n    rigid_inverse(T_ref, M);\n    const float t2",
     "    float M[16];\n    rigid_inverse(T_g, M);\n    const float t2"),
    (TRACK, "normal validity not checked", "            if (!(Vp[3] > 0.0f && Np[3] > 0.0f)) continue;",
     "            if (!(Vp[3] > 0.0f)) continue;"),
    (TRACK, "invalid depths in the pyramid mean", "                if (d > 0.0f) {\n                    sum = sum + d;",
     "                if (1) {\n                    sum = sum + d;"),
    (TRACK, "pyramid centre c/2", "    out[2] = (in[2] - 0.5f) / 2.0f;", "    out[2] = in[2] / 2.0f;"),
    (TRACK, "residual sign", "            const float res = (dx * Np[0] + dy * Np[1]) + dz * Np[2];",
     "            const float res = -((dx * Np[0] + dy * Np[1]) + dz * Np[2]);"),
    (TRACK, "threshold on the distance, not its square", "            if (!(dist2 <= t2)) continue;",
     "            if (!(dist2 <= dist_thresh)) continue;"),
    (TRACK, "Gauss-Newton right-hand side sign", "    for (int i = 0; i < 6; ++i) b[i] = -sums[21 + i];",
     "    for (int i = 0; i < 6; ++i) b[i] = sums[21 + i];"),
    (TRACK, "Cholesky divisor from the wrong row", "                L[i][j] = acc / L[j][j];",
     "                L[i][j] = acc / L[i][i];"),
    (TRACK, "Rodrigues sine sign",
     "R[i][j] = (i == j ? 1.0 : 0.0) + a * K[i][j] + c * K2[i][j];",
     "R[i][j] = (i == j ? 1.0 : 0.0) - a * K[i][j] + c * K2[i][j];"),
    (MESH, "ambiguous faces joined around outside corners", "                int want = (posA[k] + 3) & 3;",
     "                int want = (posA[k] + 1) & 3;"),
    (MESH, "fan not flipped", "            tri[3 * n_tri + 1] = loop[i + 1];\n            tri[3 * n_tri + 2] = loop[i];",
     "            tri[3 * n_tri + 1] = loop[i];\n            tri[3 * n_tri + 2] = loop[i + 1];"),
    (MESH, "crossing t from the wrong end", "                    float tt = F[a] / (F[a] - F[c]);",
     "                    float tt = F[c] / (F[c] - F[a]);"),
    (MESH, "weights not checked", "    if (!(s->w[i] > 0.0f)) return 0;\n    *F = s->sdf[i];", "    *F = s->sdf[i];"),
    (MESH, "edge numbering swapped", "    return 4 * axis + o1 + 2 * o2;", "    return 4 * axis + 2 * o1 + o2;"),
    (MESH, "a face walked clockwise", "    {0, 4, 6, 2}, {1, 3, 7, 5},", "    {0, 2, 6, 4}, {1, 3, 7, 5},"),
    (MESH, "F = 0 taken as inside", "            int ia = F[a] < 0.0f, ib = F[b] < 0.0f;",
     "            int ia = F[a] <= 0.0f, ib = F[b] <= 0.0f;"),
    (MESH, "corner z offset from the y bit",
     "                ok = observed_value(s, g[0] + (k & 1), g[1] + ((k >> 1) & 1), g[2] + (k >> 2), &F[k]);",
     "                ok = observed_value(s, g[0] + (k & 1), g[1] + ((k >> 1) & 1), g[2] + ((k >> 1) & 1), &F[k]);"),
    (MESH, "edge axes x and y swapped", "                    int axis = (c - a) == 1 ? 0 : (c - a) == 2 ? 1 : 2;",
     "                    int axis = (c - a) == 2 ? 0 : (c - a) == 1 ? 1 : 2;"),
    (MESH, "corner offset on the wrong axis", "                        float coord = (float)(g[k] + ((a >> k) & 1));",
     "                        float coord = (float)(g[k] + ((a >> ((k + 1) % 3)) & 1));"),
    # a scene split over processes by slabs of block columns
    (SHARD, "slab owner by truncation", "    int q = bx >= 0 ? bx / w : -((-bx + w - 1) / w); /* floor(bx / w) */",
     "    int q = bx / w;"),
    (SHARD, "no ghost columns", "#define ORC_SHARD_GHOST 1", "#define ORC_SHARD_GHOST 0"),
    (SHARD, "hits in other parts' columns reported",
     "            if (!shard_owns(s, ((int)floorf(q[0] + 0.5f)) >> 3)) continue; /* another part's hit */\n", ""),
    (SHARD, "merge keeps the farthest hit", "            if (best < 0 || z < best_z) {", "            if (best < 0 || z > best_z) {"),
    (SHARD, "merge ties to the higher part", "            if (best < 0 || z < best_z) {", "            if (best < 0 || z <= best_z) {"),
    (SHARD, "merge depth from the wrong row", "            const float z = row_apply(&M[8], V[0], V[1], V[2]);",
     "            const float z = row_apply(&M[4], V[0], V[1], V[2]);"),
]


def _run_mutant(root, module, mistake, old, new):
    """Plant one mistake in a copy of the oracle under root and run its pin
    module there; returns why the pins did not catch it, or None."""
    src = open(os.path.join(ROOT, "oracle", "itm_oracle.c")).read()
    if src.count(old) != 1:
        return "the planted line no longer matches the oracle once"
    for d in ("tests", "synth"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(root, d), ignore=shutil.ignore_patterns("__pycache__"))
    os.mkdir(os.path.join(root, "oracle"))
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), os.path.join(root, "oracle", "__init__.py"))
    with open(os.path.join(root, "oracle", "itm_oracle.c"), "w") as f:
        f.write(src.replace(old, new))
    # the pin modules need no GPU check (and so no torch import) in the copy
    with open(os.path.join(root, "tests", "conftest.py"), "w") as f:
        f.write("import os, sys\nsys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))\n")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "tests/" + module],
                       cwd=root, capture_output=True, text=True, timeout=900)
    if r.returncode == 0:
        return "the pins did not catch it"
    if "assert" not in r.stdout:
        return "failed for another reason than an assertion:\n" + r.stdout[-1500:]
    return None


def test_every_planted_mistake_fails_a_pin(tmp_path):
    """Each mistake in its own copy, the copies run side by side on the host's
    cores (they share nothing)."""
    from concurrent.futures import ThreadPoolExecutor
    assert len({m[1] for m in MUTANTS}) == len(MUTANTS)
    workers = max(1, min(len(MUTANTS), os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as pool:
        futs = [pool.submit(_run_mutant, str(tmp_path / ("m%03d" % i)), *m) for i, m in enumerate(MUTANTS)]
        escaped = [(m[0], m[1], f.result()) for m, f in zip(MUTANTS, futs) if f.result() is not None]
    assert not escaped, escaped
