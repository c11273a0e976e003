"""Mutation sweep of the C oracle (run by hand: python tests/oracle_mutants.py).

Each entry plants one plausible mistake in oracle/ad_oracle.c (or in the
argument conversions of its Python binding, oracle/__init__.py) -- a swapped
operand, a dropped term, a wrong index, sign or constant, an off-by-one -- then
rebuilds the oracle and runs the CPU suite (pytest -m "not gpu").  A mistake
that no test catches marks a weak pin.  The source is restored (and the oracle
rebuilt) after every mutant and on any exit.

Three mutants are equivalent and are expected to survive:
  target_min0  the clamp T >= 1 never acts: d >= 1 and e >= 0 give d^e >= 1;
  grad_A_sign  the rescale term it changes is multiplied by sum_i dL/dx_i, which
               is zero for a loss of distances (shifting every x leaves L unchanged);
  upward_rescale_once  rescaling once after the sweeps equals rescaling after
               every sweep in exact arithmetic (the sweep commutes with affine maps).
"""
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, 'oracle', 'ad_oracle.c')
PY_SRC = os.path.join(ROOT, 'oracle', '__init__.py')
EQUIVALENT = {'target_min0', 'grad_A_sign', 'upward_rescale_once'}

M = [
    # Philox and init
    ('philox_key_mix', 'uint32_t n0 = hi1 ^ c1 ^ k0;', 'uint32_t n0 = hi1 ^ c1 ^ k1;', 0),
    ('philox_bump_swap', 'if (round > 0) { k0 += W0; k1 += W1; }', 'if (round > 0) { k0 += W1; k1 += W0; }', 0),
    ('philox_rounds9', 'for (int round = 0; round < 10; ++round)', 'for (int round = 0; round < 9; ++round)', 0),
    ('init_ctr_r_mod', 'ctr[2] = (uint32_t)(r / 4);', 'ctr[2] = (uint32_t)(r % 4);', 0),
    ('init_word_shift', 'uint32_t u = out[r % 4];', 'uint32_t u = out[(r + 1) % 4];', 0),
    ('init_offset', '* (1.0 / 16777216.0) - 0.5;', '* (1.0 / 16777216.0) - 0.25;', 0),
    ('init_scale', '(double)(u >> 8) * (1.0 / 16777216.0)', '(double)(u >> 9) * (1.0 / 16777216.0)', 0),
    ('init_ctr_hi', 'ctr[1] = (uint32_t)((uint64_t)i >> 32);', 'ctr[1] = (uint32_t)((uint64_t)i & 1);', 0),
    ('init_stream_ignored', 'ctr[3] = stream;', 'ctr[3] = 0;', 0),
    ('init_key_hi_dropped', 'key[1] = (uint32_t)(seed >> 32);', 'key[1] = 0;', 0),
    # degrees, sweep, rescale, distance
    ('degree_ignores_w', 's += (w ? w[p] : 1.0);\n        D[i] = s;', 's += 1.0;\n        D[i] = s;', 0),
    ('sweep_alpha_swap', 'y[i] = alpha * x[i] + (1.0 - alpha) * s / D[i];', 'y[i] = (1.0 - alpha) * x[i] + alpha * s / D[i];', 0),
    ('sweep_wrong_neighbour', 's += (w ? w[p] : 1.0) * x[ci[p]];', 's += (w ? w[p] : 1.0) * x[i];', 0),
    ('sweep_drops_weight', 's += (w ? w[p] : 1.0) * x[ci[p]];', 's += x[ci[p]];', 0),
    ('rescale_counts_inactive', '        if (!(D[i] > 0.0)) continue;\n        if (x[i] < lo) lo = x[i];', '        if (x[i] < lo) lo = x[i];', 0),
    ('rescale_centre', 'x[i] = (hi > lo) ? (x[i] - lo) / (hi - lo) - 0.5 : 0.0;', 'x[i] = (hi > lo) ? (x[i] - lo) / (hi - lo) - 0.4 : 0.0;', 0),
    ('rescale_degenerate', 'x[i] = (hi > lo) ? (x[i] - lo) / (hi - lo) - 0.5 : 0.0;', 'x[i] = (hi > lo) ? (x[i] - lo) / (hi - lo) - 0.5 : x[i];', 0),
    ('rescale_denominator', 'x[i] = (hi > lo) ? (x[i] - lo) / (hi - lo) - 0.5 : 0.0;', 'x[i] = (hi > lo) ? (x[i] - lo) / (hi) - 0.5 : 0.0;', 0),
    ('dist_l1', 'acc[e] += d * d;', 'acc[e] += fabs(d);', 0),
    ('dist_no_sqrt', 'double s = sqrt(acc[e]);', 'double s = acc[e];', 0),
    ('dist_normalize_wrong_end', 'if (normalize) s *= sqrt(D[i] * D[ci[p]]);', 'if (normalize) s *= sqrt(D[i] * D[i]);', 0),
    ('sweep_count_off_by_one', 'for (int32_t t = 0; t < k; ++t) {', 'for (int32_t t = 0; t < k - 1; ++t) {', 0),
    # selection
    ('asc_tie_reversed', 'if (x->s > y->s) return 1;\n    return (x->e < y->e) ? -1 : (x->e > y->e);', 'if (x->s > y->s) return 1;\n    return (x->e > y->e) ? -1 : (x->e < y->e);', 0),
    ('desc_tie_reversed', 'if (x->s < y->s) return 1;\n    return (x->e < y->e) ? -1 : (x->e > y->e);', 'if (x->s < y->s) return 1;\n    return (x->e > y->e) ? -1 : (x->e < y->e);', 0),
    ('target_floor', 'double t = ceil(pow((double)d, e) - 1e-9);', 'double t = floor(pow((double)d, e) - 1e-9);', 0),
    ('target_min0', 'if (t < 1.0) t = 1.0;', 'if (t < 0.0) t = 0.0;', 0),
    ('target_eps_sign', 'double t = ceil(pow((double)d, e) - 1e-9);', 'double t = ceil(pow((double)d, e) + 1e-9);', 0),
    ('K_no_round', 'return (int64_t)floor(fraction * (double)m + 0.5);', 'return (int64_t)floor(fraction * (double)m);', 0),
    ('bisect_strict_alg2', 'if (union_of_tops(n, rp, sorted_e, m, mid, keep) >= K) hi = mid; else lo = mid;', 'if (union_of_tops(n, rp, sorted_e, m, mid, keep) > K) hi = mid; else lo = mid;', 0),
    ('bisect_strict_binned', 'if (union_of_tops(n, rp, sorted_e, m, mid, keep) >= K) hi = mid; else lo = mid;', 'if (union_of_tops(n, rp, sorted_e, m, mid, keep) > K) hi = mid; else lo = mid;', 1),
    ('bisect_strict_ld', 'if (union_of_tops(n, rp, sorted_e, m, mid, keep) >= K) hi = mid; else lo = mid;', 'if (union_of_tops(n, rp, sorted_e, m, mid, keep) > K) hi = mid; else lo = mid;', 2),
    ('union_off_by_one', 'for (int64_t t = 0; t < T; ++t) keep[sorted_e[rp[i] + t]] = 1;', 'for (int64_t t = 0; t + 1 < T; ++t) keep[sorted_e[rp[i] + t]] = 1;', 0),
    ('whole_graph_K_minus_1', 'for (int64_t t = 0; t < K; ++t) keep[a[t].e] = 1;', 'for (int64_t t = 0; t + 1 < K; ++t) keep[a[t].e] = 1;', 0),
    ('per_node_mode_swapped', 'qsort(a, (size_t)d, sizeof(scored_edge), mode ? cmp_descending : cmp_ascending);', 'qsort(a, (size_t)d, sizeof(scored_edge), mode ? cmp_ascending : cmp_descending);', 0),
    # SparsifyB
    ('binned_sample_sigma', 'const float sigma = sqrtf(q / (float)d);', 'const float sigma = sqrtf(q / (float)(d > 1 ? d - 1 : 1));', 0),
    ('binned_scott_const', 'const float h = 3.5f * sigma', 'const float h = 3.0f * sigma', 0),
    ('binned_sqrt_not_cbrt', '(float)cbrt((double)d)', '(float)sqrt((double)d)', 0),
    ('binned_no_min_shift', 'b = (int64_t)floorf(((float)score[eid[p0 + t]] - lo) / h);', 'b = (int64_t)floorf(((float)score[eid[p0 + t]]) / h);', 0),
    ('binned_word_by_position', 'a[t].u = bin_word(seed, (uint64_t)eid[p0 + t], 0u);', 'a[t].u = bin_word(seed, (uint64_t)(p0 + t), 0u);', 0),
    ('binned_bin_word_index', 'bk[b].v = bin_word(seed, (uint64_t)i, (uint32_t)(1 + b));', 'bk[b].v = bin_word(seed, (uint64_t)i, (uint32_t)(b));', 0),
    ('binned_round_order', 'if (size[c] > r && order[c] < order[b]) ++rk;', 'if (size[c] > r && order[c] > order[b]) ++rk;', 0),
    ('binned_stream', '#define ORC_BIN_STREAM 0xB1000000u', '#define ORC_BIN_STREAM 0xB1000001u', 0),
    ('binned_within_desc', 'if (x->u != y->u) return x->u < y->u ? -1 : 1;', 'if (x->u != y->u) return x->u > y->u ? -1 : 1;', 0),
    # Local Degree
    ('ld_degree_ascending', 'if (x->d != y->d) return x->d > y->d ? -1 : 1;', 'if (x->d != y->d) return x->d < y->d ? -1 : 1;', 0),
    # multilevel
    ('seeds_order_ascending', 'if (x->D > y->D) return -1;\n    if (x->D < y->D) return 1;', 'if (x->D < y->D) return -1;\n    if (x->D > y->D) return 1;', 0),
    ('seeds_strict_Q', 'if (to_seeds <= Q * D[i]) is_seed[i] = 1;', 'if (to_seeds < Q * D[i]) is_seed[i] = 1;', 0),
    ('seeds_ignore_w', 'if (is_seed[ci[p]]) to_seeds += (w ? w[p] : 1.0);', 'if (is_seed[ci[p]]) to_seeds += 1.0;', 0),
    ('agg_argmax', 'if (best < 0 || s < best_s || (s == best_s && j < best))', 'if (best < 0 || s > best_s || (s == best_s && j < best))', 0),
    ('agg_tie_larger', 'if (best < 0 || s < best_s || (s == best_s && j < best))', 'if (best < 0 || s < best_s || (s == best_s && j > best))', 0),
    ('galerkin_overwrite', 'uw[mc - 1] += pairs[t].w;', 'uw[mc - 1] = pairs[t].w;', 0),
    ('uncoarsen_drop_intra', 'keep_f[e] = (fine_to_coarse[e] < 0) ? 1 : keep_c[fine_to_coarse[e]];', 'keep_f[e] = (fine_to_coarse[e] < 0) ? 0 : keep_c[fine_to_coarse[e]];', 0),
    ('stall_guard', 'if ((double)nc > 0.9 * (double)cn)', 'if ((double)nc > 0.5 * (double)cn)', 0),
    ('level_stream_down', '(uint32_t)(2 * l),', '(uint32_t)(l),', 0),
    ('level_stream_up', '(uint32_t)(2 * l + 1)', '(uint32_t)(2 * l)', 0),
    ('segment_middle', 'else if (segment == 2) start = (L - s) / 2;', 'else if (segment == 2) start = (L - s + 1) / 2;', 0),
    ('ratios_not_reversed', 'for (int32_t l = 0; l < L; ++l) r_by_level[l] = ratios[L - 1 - l];', 'for (int32_t l = 0; l < L; ++l) r_by_level[l] = ratios[l];', 0),
    # reverse mode
    ('grad_loss_factor', 'xbar[eu[e]] += 2.0 * d;', 'xbar[eu[e]] += d;', 0),
    ('grad_A_sign', 'A += xbar[i] * (x[i] - 0.5);', 'A += xbar[i] * (x[i] + 0.5);', 0),
    ('grad_B_sign', 'ybar[amax[t]] -= a[t] * B;', 'ybar[amax[t]] += a[t] * B;', 0),
    ('grad_drop_avg', 'gentry[p] += ybar[i] * omega * (xp[ci[p]] - avg) / D[i];', 'gentry[p] += ybar[i] * omega * (xp[ci[p]]) / D[i];', 0),
    ('grad_alpha_omega', 'xbar[j] = alpha * ybar[j] + s;', 'xbar[j] = omega * ybar[j] + s;', 0),
    ('grad_transposed_D', 's += ybar[i] * omega * (w ? w[p] : 1.0) / D[i];', 's += ybar[i] * omega * (w ? w[p] : 1.0) / D[j];', 0),
    # second batch: Galerkin, kept subgraph, upward pass, fit, Local Degree key, init layout
    ('galerkin_not_canonical', 'pairs[np].a = I < J ? I : J; pairs[np].b = I < J ? J : I;', 'pairs[np].a = I; pairs[np].b = J;', 0),
    ('galerkin_drops_w', 'pairs[np].fe = e; pairs[np].w = w ? w[p] : 1.0; ++np;', 'pairs[np].fe = e; pairs[np].w = 1.0; ++np;', 0),
    ('kept_subgraph_drops_w', 'ci_s[q] = ci[p]; w_s[q] = w ? w[p] : 1.0; ++q;', 'ci_s[q] = ci[p]; w_s[q] = 1.0; ++q;', 0),
    ('coarsest_starts_empty', 'for (int64_t e = 0; e < v->m; ++e) keep[e] = 1;', 'for (int64_t e = 0; e < v->m; ++e) keep[e] = 0;', 0),
    ('levels_stop_strict', 'if (cn <= coarsest_n || l + 1 >= max_levels) break;', 'if (cn < coarsest_n || l + 1 >= max_levels) break;', 0),
    ('ml_fit_19_halvings', 'for (int it = 0; it < 20; ++it) {', 'for (int it = 0; it < 19; ++it) {', 0),
    ('alg2_returns_lo', '    *n_kept = union_of_tops(n, rp, sorted_e, m, hi, keep);\n    *e_used = hi;\n    free(sorted_e);', '    *n_kept = union_of_tops(n, rp, sorted_e, m, lo, keep);\n    *e_used = lo;\n    free(sorted_e);', 0),
    ('ld_key_is_id', 'a[t].d = rp[j + 1] - rp[j];', 'a[t].d = j;', 0),
    ('init_layout_transposed', 'x[i * R + r] = orc_test_value(seed, stream, i, r);', 'x[r * n + i] = orc_test_value(seed, stream, i, r);', 0),
    ('whole_graph_mode_swapped', 'qsort(a, (size_t)m, sizeof(scored_edge), mode ? cmp_descending : cmp_ascending);', 'qsort(a, (size_t)m, sizeof(scored_edge), mode ? cmp_ascending : cmp_descending);', 0),
    ('normalize_divides', 'if (normalize) s *= sqrt(D[i] * D[ci[p]]);', 'if (normalize) s /= sqrt(D[i] * D[ci[p]]);', 0),
    ('upward_rescale_once', '(uint32_t)(2 * l + 1), 0, 0, NULL, NULL, rhos)', '(uint32_t)(2 * l + 1), 1, 0, NULL, NULL, rhos)', 0),
    ('seed_numbering_all', 'for (int64_t i = 0; i < n; ++i) agg[i] = is_seed[i] ? (int32_t)(nc++) : -1;', 'for (int64_t i = n - 1; i >= 0; --i) agg[i] = is_seed[i] ? (int32_t)(nc++) : -1;', 0),
]



# mistakes in the Python binding of the oracle (argument conversions)
PY_M = [
    ('py_alpha_not_converted', 'R, k, 1.0 - omega,\n                                     seed, stream, mode,', 'R, k, omega,\n                                     seed, stream, mode,', 0),
    ('py_ml_alpha_not_converted', 'R, k, 1.0 - omega, seed, Q, coarsest_n,', 'R, k, omega, seed, Q, coarsest_n,', 0),
    ('py_grad_alpha_not_converted', 'R, k, 1.0 - omega, seed,\n                            stream,', 'R, k, omega, seed,\n                            stream,', 0),
    ('py_modes_swapped', 'MODES = {"local": 0, "global": 1}', 'MODES = {"local": 1, "global": 0}', 0),
    ('py_scopes_swapped', 'SCOPES = {"per_node": 0, "whole_graph": 1}', 'SCOPES = {"per_node": 1, "whole_graph": 0}', 0),
    ('py_rescale_modes_swapped', 'mode = {"per_sweep": 0, "end": 1}[rescale]', 'mode = {"per_sweep": 1, "end": 0}[rescale]', 0),
]


def nth_replace(s, old, new, k):
    idx = -1
    for _ in range(k + 1):
        idx = s.find(old, idx + 1)
        if idx < 0:
            raise ValueError('occurrence %d not found' % k)
    return s[:idx] + new + s[idx + len(old):]


def rebuild():
    r = subprocess.run([sys.executable, '-c', 'import oracle; oracle.build(force=True)'], cwd=ROOT,
                       capture_output=True, text=True)
    return r.returncode == 0, r.stderr[-400:]


def main():
    only = sys.argv[1:]
    orig = open(SRC).read()
    backup = os.path.join(tempfile.mkdtemp(prefix='oracle_mutants_'), 'ad_oracle.c')
    shutil.copy(SRC, backup)
    res = {}
    py_orig = open(PY_SRC).read()
    try:
        for name, old, new, k in PY_M:
            if only and name not in only:
                continue
            if py_orig.count(old) <= k:
                res[name] = 'pattern missing'
                print(name, res[name], flush=True)
                continue
            with open(PY_SRC, 'w') as f:
                f.write(nth_replace(py_orig, old, new, k))
            r = subprocess.run([sys.executable, '-m', 'pytest', 'tests', '-m', 'not gpu', '-x', '-q',
                                '-p', 'no:cacheprovider'], cwd=ROOT, capture_output=True, text=True, timeout=900)
            with open(PY_SRC, 'w') as f:
                f.write(py_orig)
            res[name] = 'killed' if r.returncode != 0 else 'survived'
            first = [l for l in r.stdout.splitlines() if l.startswith('FAILED')][:1]
            print(name, res[name], first[0][:110] if first else '', flush=True)
        for name, old, new, k in M:
            if only and name not in only:
                continue
            if orig.count(old) <= k:
                res[name] = 'pattern missing'
                print(name, res[name], flush=True)
                continue
            with open(SRC, 'w') as f:
                f.write(nth_replace(orig, old, new, k))
            ok, err = rebuild()
            if not ok:
                res[name] = 'build failed'
                print(name, res[name], err, flush=True)
                continue
            r = subprocess.run([sys.executable, '-m', 'pytest', 'tests', '-m', 'not gpu', '-x', '-q',
                                '-p', 'no:cacheprovider'], cwd=ROOT, capture_output=True, text=True, timeout=900)
            res[name] = 'killed' if r.returncode != 0 else 'survived'
            first = [l for l in r.stdout.splitlines() if l.startswith('FAILED')][:1]
            print(name, res[name], first[0][:110] if first else '', flush=True)
    finally:
        with open(PY_SRC, 'w') as f:
            f.write(py_orig)
        with open(SRC, 'w') as f:
            f.write(orig)
        rebuild()
    weak = [k for k, v in res.items() if v != 'killed' and k not in EQUIVALENT]
    print('%d mutants, %d killed; equivalent survivors: %s; weak pins: %s'
          % (len(res), sum(v == 'killed' for v in res.values()),
             sorted(k for k in res if k in EQUIVALENT and res[k] != 'killed'), weak or 'none'))
    return 1 if weak else 0


if __name__ == '__main__':
    sys.exit(main())
