// PTX guard pass (Sec. V-E): parse application PTX, insert the kernel memory guard
// before every global-memory access, and serialize the result for loading.
//
// What is guarded: ld, ldu, st, atom and red on the .global state space, and on the
// generic space when the address resolves to global memory (isspacep.global). Shared,
// local, const and param accesses are left alone. Functions named in the skip list
// (trusted module bodies, Sec. V-E) are left untouched. Forms the guard cannot cover --
// bulk and tensor copies (cp.*), asynchronous stores/reductions, multimem, surfaces,
// tensormap and discard -- are rejected (fail closed, Sec. IV-C).
//
// The inserted sequence, per access of W bytes at effective address a, in program order:
//   1. inline bitmap test: the all-user bitmap's word for a's block, and the first and
//      last byte of the access in the same block;
//   2. when the bitmap block is mixed, inline class-map test: a's block in the 2-bit block
//      class map is class 1 (inside one user range) and holds the whole access;
//   3. only then the slow path, inlined with labels of its own: the page map, else the
//      binary search over the page's ranges and the walk (full classification). A
//      denial is appended to the log's bounded list when one is attached, and counted:
//      in the registers of an entry function (merged per warp by __agile_guard_flush
//      before each ret and exit), else merged into the log at once;
//   then the policy: POISON/SINK send a denied load to the zero page; POISON predicates
//   a denied store/atom/red off (a denied atom's result reads 0), SINK sends it to the
//   sink page; REPORT changes nothing; TRAP emits `@!ok trap;`.
// The table's device address is read once per function from the module global
// __agile_guard_table; site = the access's position in its function.
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <set>
#include <string>
#include <vector>

#include "agile_internal.h"
#include "ptx_guard_check.inc"

namespace {

// The injected PTX reads the table header by byte offset.
static_assert(offsetof(agile_dev_table_t, lo) == 0 && offsetof(agile_dev_table_t, n) == 20 &&
                  offsetof(agile_dev_table_t, base) == 32 && offsetof(agile_dev_table_t, end) == 40 &&
                  offsetof(agile_dev_table_t, kind) == 48 && offsetof(agile_dev_table_t, id) == 56 &&
                  offsetof(agile_dev_table_t, zero_page) == 64 &&
                  offsetof(agile_dev_table_t, sink_page) == 72 &&
                  offsetof(agile_dev_table_t, remap_or) == 104 &&
                  offsetof(agile_dev_table_t, ubits) == 112 &&
                  offsetof(agile_dev_table_t, ubits_log2) == 120 &&
                  offsetof(agile_dev_table_t, ubits_n) == 124,
              "header offsets used by the injected PTX");

struct Fail {
    int code;
};

bool is_ident_start(char c) { return std::isalpha((unsigned char)c) || c == '_' || c == '$' || c == '%'; }
bool is_ident(char c) { return std::isalnum((unsigned char)c) || c == '_' || c == '$'; }

std::string trim(const std::string &s) {
    size_t a = 0, b = s.size();
    while (a < b && std::isspace((unsigned char)s[a])) ++a;
    while (b > a && std::isspace((unsigned char)s[b - 1])) --b;
    return s.substr(a, b - a);
}

// Copy of `s` with comments and string literals blanked to spaces (same length), so
// that positions found in the clean text index the raw text.
std::string blank_comments(const std::string &s) {
    std::string c = s;
    size_t i = 0, n = s.size();
    while (i < n) {
        if (s[i] == '/' && i + 1 < n && s[i + 1] == '/') {
            while (i < n && s[i] != '\n') c[i++] = ' ';
        } else if (s[i] == '/' && i + 1 < n && s[i + 1] == '*') {
            size_t e = s.find("*/", i + 2);
            if (e == std::string::npos) throw Fail{AGILE_ERR_PTX_PARSE};
            for (; i < e + 2; ++i) if (c[i] != '\n') c[i] = ' ';
        } else if (s[i] == '"') {
            size_t e = s.find('"', i + 1);
            if (e == std::string::npos) throw Fail{AGILE_ERR_PTX_PARSE};
            for (++i; i < e; ++i) c[i] = ' ';
            ++i;
        } else {
            ++i;
        }
    }
    return c;
}

int type_bytes(const std::string &t) {
    static const char *b1[] = {"b8", "u8", "s8"};
    static const char *b2[] = {"b16", "u16", "s16", "f16", "bf16"};
    static const char *b4[] = {"b32", "u32", "s32", "f32", "f16x2", "bf16x2"};
    static const char *b8[] = {"b64", "u64", "s64", "f64"};
    for (auto x : b1) if (t == x) return 1;
    for (auto x : b2) if (t == x) return 2;
    for (auto x : b4) if (t == x) return 4;
    for (auto x : b8) if (t == x) return 8;
    if (t == "b128") return 16;
    return 0;
}

std::vector<std::string> split_dots(const std::string &op) {
    std::vector<std::string> out;
    size_t i = 0;
    while (i <= op.size()) {
        size_t j = op.find('.', i);
        // "::" qualifiers stay attached to their modifier
        if (j == std::string::npos) j = op.size();
        out.push_back(op.substr(i, j - i));
        i = j + 1;
    }
    return out;
}

struct Access {
    enum Kind { LOAD, STORE, ATOM, RED } kind;
    bool generic = false;
    int width = 0;
    int dest_bits = 0;          // atom: scalar result size, 0 if not zeroable
    std::string dest;
};

// One aperture in decision order (MMIO before protected, then by base).
struct Aperture {
    uint64_t lo, end;
    uint32_t verdict, id;
};

class Rewriter {
  public:
    Rewriter(int policy, const std::set<std::string> &skip, std::vector<Aperture> aps, bool aperture)
        : policy_(policy), skip_(skip), aps_(std::move(aps)), aperture_(aperture) {
        if (aperture_ && !aps_.empty()) {
            hull_lo_ = aps_[0].lo;
            hull_end_ = aps_[0].end;
            for (const Aperture &a : aps_) {
                hull_lo_ = std::min(hull_lo_, a.lo);
                hull_end_ = std::max(hull_end_, a.end);
            }
        }
        injected_ = std::string(kGuardGlobalsPtx);
        if (aperture_) {
            injected_ += kApertureGlobalsPtx;
            injected_ += ".global .align 4 .u32 __agile_aperture_mode = 1;\n";
        }
        injected_ += kGuardLogPtx;
        injected_ += kGuardFlushPtx;
        // The slow path inlined at each access: classification, then the info word in
        // %t16 (0 when allowed), registers renamed into the pass's own namespace.
        slow_ = rename_regs((aperture_ ? aperture_body() : std::string(kGuardCheckTablePtx)) +
                            "$AGC_LOG:\n" + kGuardInfoPtx +
                            "\tbra.uni $AGC_END;\n$AGC_RET:\n\tmov.b64 %t16, 0;\n$AGC_END:\n");
    }

    std::string run(const std::string &ptx) {
        if (ptx.find("__ag") != std::string::npos) throw Fail{AGILE_ERR_PTX_UNSUPPORTED};
        const std::string clean = blank_comments(ptx);
        size_t as = clean.find(".address_size");
        if (as == std::string::npos) throw Fail{AGILE_ERR_PTX_UNSUPPORTED};
        {
            size_t k = as + 13;
            while (k < clean.size() && std::isspace((unsigned char)clean[k])) ++k;
            if (clean.compare(k, 2, "64") != 0) throw Fail{AGILE_ERR_PTX_UNSUPPORTED};
        }
        // Entry functions keep their violations in registers and merge them before they
        // exit, unless a trap may end the kernel before that (TRAP policy) or a called
        // function may exit the thread with the entry's registers unmerged.
        acc_module_ = policy_ != AGILE_POLICY_TRAP && !func_may_exit(clean);
        size_t inject_at = clean.find('\n', as);
        if (inject_at == std::string::npos) inject_at = clean.size();

        std::string out;
        out.reserve(ptx.size() * 3);
        size_t i = 0, n = clean.size(), stmt_start = 0;
        bool injected = false;
        while (i < n) {
            if (!injected && i >= inject_at) {
                out.append(ptx, stmt_start, i - stmt_start);
                out += "\n";
                out += injected_;
                stmt_start = i;
                injected = true;
            }
            char ch = clean[i];
            if (ch == ';') {
                ++i;
                out.append(ptx, stmt_start, i - stmt_start);
                stmt_start = i;
            } else if (ch == '{') {
                size_t close = match_brace(clean, i);
                std::string header = clean.substr(stmt_start, i - stmt_start);
                out.append(ptx, stmt_start, i - stmt_start);
                if (is_function_header(header)) {
                    std::string body = ptx.substr(i + 1, close - i - 1);
                    std::string name = function_name(header);
                    ++rep_.functions;
                    out += "{";
                    out += rewrite_body(body, skip_.count(name) != 0, has_token(header, ".entry"));
                    out += "}";
                } else {
                    out.append(ptx, i, close - i + 1);
                }
                i = close + 1;
                stmt_start = i;
            } else if (ch == '}') {
                throw Fail{AGILE_ERR_PTX_PARSE};
            } else {
                ++i;
            }
        }
        out.append(ptx, stmt_start, n - stmt_start);
        if (!injected) out += injected_;
        // Fail closed: every memory-access opcode word of the input must have been seen
        // by the statement parser (guarded, skipped, or on a non-global space).
        if (count_access_words(clean) != rep_.guarded + rep_.skipped + other_space_)
            throw Fail{AGILE_ERR_PTX_PARSE};
        return out;
    }

    agile_instrument_report_t rep_{};

  private:
    uint32_t other_space_ = 0;

    // True when the body of some .func holds the word "exit" (read as the instruction).
    static bool func_may_exit(const std::string &clean) {
        size_t i = 0, n = clean.size(), stmt_start = 0;
        while (i < n) {
            const char ch = clean[i];
            if (ch == ';') {
                stmt_start = ++i;
            } else if (ch == '{') {
                const size_t close = match_brace(clean, i);
                if (has_token(clean.substr(stmt_start, i - stmt_start), ".func") &&
                    has_word(clean.substr(i, close - i), "exit"))
                    return true;
                i = close + 1;
                stmt_start = i;
            } else {
                ++i;
            }
        }
        return false;
    }

    // `w` as a whole word: not part of an identifier, a directive, a register or a label.
    static bool has_word(const std::string &t, const char *w) {
        const size_t L = std::strlen(w);
        for (size_t p = t.find(w); p != std::string::npos; p = t.find(w, p + 1)) {
            const bool left = p == 0 || !(is_ident(t[p - 1]) || t[p - 1] == '.' || t[p - 1] == '%' ||
                                          t[p - 1] == '$');
            const bool right = p + L >= t.size() || !is_ident(t[p + L]);
            if (left && right) return true;
        }
        return false;
    }

    // Independent count of ld/ldu/st/atom/red opcode words, by a plain word scan.
    static uint32_t count_access_words(const std::string &clean) {
        uint32_t c = 0;
        size_t i = 0, n = clean.size();
        while (i < n) {
            if (std::isalpha((unsigned char)clean[i]) &&
                (i == 0 || !(is_ident(clean[i - 1]) || clean[i - 1] == '.' || clean[i - 1] == '%'))) {
                size_t e = i;
                while (e < n && is_ident(clean[e])) ++e;
                std::string w = clean.substr(i, e - i);
                if (e < n && clean[e] == '.' &&
                    (w == "ld" || w == "ldu" || w == "st" || w == "atom" || w == "red"))
                    ++c;
                i = e;
            } else {
                ++i;
            }
        }
        return c;
    }

    int policy_;
    const std::set<std::string> &skip_;
    std::vector<Aperture> aps_;
    bool aperture_;
    uint64_t hull_lo_ = 0, hull_end_ = 0;   // smallest interval holding every aperture
    std::string injected_;
    std::string slow_;          // the inlined slow path, labels still $AGC_
    int label_ = 0;
    bool acc_module_ = false;   // entries of this module keep violations in registers
    bool acc_fn_ = false;       // ... and the function being rewritten is one of them

    // %t<k>, %s<k>, %q<k> of the slow-path template become %__agt<k>, %__ags<k>, %__agq<k>.
    static std::string rename_regs(const std::string &t) {
        std::string o;
        o.reserve(t.size() + t.size() / 4);
        for (size_t i = 0; i < t.size(); ++i) {
            o += t[i];
            if (t[i] == '%' && i + 2 < t.size() && (t[i + 1] == 't' || t[i + 1] == 's' || t[i + 1] == 'q') &&
                std::isdigit((unsigned char)t[i + 2]))
                o += "__ag";
        }
        return o;
    }

    // The slow path for the access at `addr` (a 64-bit register) of `width` bytes at
    // `site`, with labels of its own; leaves the info word in %__agt16, 0 when allowed.
    std::string inline_check(const std::string &addr, const std::string &width, int site) {
        const std::string tag = "$__AGC" + std::to_string(label_++) + "_";
        std::string body = slow_;
        for (size_t p = body.find("$AGC_"); p != std::string::npos; p = body.find("$AGC_", p + tag.size()))
            body.replace(p, 5, tag);
        return "\tmov.b64 %__agt0, " + addr + ";\n\tmov.u32 %__ags0, " + width + ";\n"
               "\tmov.u32 %__ags1, " + std::to_string(site) + ";\n\tcvt.u64.u32 %__agt1, %__ags0;\n" + body;
    }

    static std::string hex(uint64_t v) {
        char b[24];
        std::snprintf(b, sizeof b, "0x%llx", (unsigned long long)v);
        return b;
    }

    // Classification under the aperture rule, the apertures as constants: INVALID as in
    // the table rule, else the first aperture (in decision order) the access overlaps.
    std::string aperture_body() const {
        std::string g =
            "    mov.u32 %s2, 5;\n"
            "    mov.u32 %s3, 0xFFFFFFFF;\n"
            "    mov.b64 %t3, 0xFFFFFFFFFFFFFFFF;\n"
            "    sub.s64 %t3, %t3, %t1;\n"
            "    setp.gt.u64 %q0, %t0, %t3;\n"
            "    setp.eq.u32 %q1, %s0, 0;\n"
            "    or.pred %q0, %q0, %q1;\n"
            "    @%q0 bra $AGC_LOG;\n"
            "    add.s64 %t4, %t0, %t1;\n"
            "    mov.u32 %s2, 0;\n";
        for (size_t k = aps_.size(); k-- > 0;) {     // the lowest index overlapped wins
            const Aperture &a = aps_[k];
            g += "    setp.lt.u64 %q1, %t0, " + hex(a.end) + ";\n"
                 "    setp.gt.and.u64 %q1, %t4, " + hex(a.lo) + ", %q1;\n"
                 "    selp.u32 %s2, " + std::to_string(a.verdict) + ", %s2, %q1;\n"
                 "    selp.u32 %s3, " + std::to_string(a.id) + ", %s3, %q1;\n";
        }
        g += "    setp.eq.u32 %q2, %s2, 0;\n"
             "    @%q2 bra $AGC_RET;\n";
        return g;
    }

    static size_t match_brace(const std::string &clean, size_t open) {
        int depth = 0;
        for (size_t k = open; k < clean.size(); ++k) {
            if (clean[k] == '{') ++depth;
            else if (clean[k] == '}' && --depth == 0) return k;
        }
        throw Fail{AGILE_ERR_PTX_PARSE};
    }

    static bool has_token(const std::string &h, const char *tok) {
        size_t p = 0, L = std::strlen(tok);
        while ((p = h.find(tok, p)) != std::string::npos) {
            bool left = p == 0 || std::isspace((unsigned char)h[p - 1]);
            bool right = p + L >= h.size() || !is_ident(h[p + L]);
            if (left && right) return true;
            p += L;
        }
        return false;
    }

    static bool is_function_header(const std::string &h) {
        return has_token(h, ".entry") || has_token(h, ".func");
    }

    static std::string function_name(const std::string &h) {
        std::string flat;
        int depth = 0;
        for (char c : h) {
            if (c == '(') ++depth;
            else if (c == ')') { --depth; flat += ' '; }
            else if (depth == 0) flat += c;
        }
        size_t k = 0;
        bool after_kw = false;
        while (k < flat.size()) {
            while (k < flat.size() && std::isspace((unsigned char)flat[k])) ++k;
            size_t e = k;
            while (e < flat.size() && !std::isspace((unsigned char)flat[e])) ++e;
            std::string tok = flat.substr(k, e - k);
            if (tok == ".entry" || tok == ".func") after_kw = true;
            else if (after_kw && !tok.empty() && tok[0] != '.') return tok;
            k = e;
        }
        return "";
    }

    std::string prologue() const {
        // Registers of an accumulating function: count, smallest (key, info).
        const std::string acc = !acc_fn_ ? std::string()
            : "\t.reg .b32 %__agc;\n\t.reg .b64 %__agk;\n\t.reg .b64 %__agi;\n"
              "\tmov.u32 %__agc, 0;\n\tmov.b64 %__agk, 0xFFFFFFFFFFFFFFFF;\n"
              "\tmov.b64 %__agi, 0xFFFFFFFFFFFFFFFF;\n";
        const std::string slow = "\t.reg .b64 %__agt<24>;\n\t.reg .b32 %__ags<20>;\n\t.reg .pred %__agq<8>;\n";
        if (aperture_)
            return "\n\t.reg .b64 %__agT<8>;\n\t.reg .b64 %__agd<8>;\n" + slow +
                   "\t.reg .b32 %__agr<3>;\n\t.reg .pred %__agp<5>;\n"
                   "\tmov.u64 %__agT3, __agile_zero_page;\n"
                   "\tmov.u64 %__agT4, __agile_sink_page;\n" + acc;
        // The fast test reads the all-user block bitmap: T0 = window start, T1 = blocks
        // in the window, T2 = bitmap, lg = log2 of the block size (header offsets 0, 124,
        // 112, 120); T3, T4 = zero and sink pages, T7 = the table.
        return "\n\t.reg .b64 %__agT<8>;\n\t.reg .b32 %__agTlg;\n\t.reg .b64 %__agd<8>;\n" + slow +
               "\t.reg .b32 %__agr<3>;\n\t.reg .pred %__agp<5>;\n"
               "\tld.global.u64 %__agT7, [__agile_guard_table];\n"
               "\tld.global.u64 %__agT0, [%__agT7];\n"
               "\tld.global.u32 %__agr0, [%__agT7+124];\n"
               "\tcvt.u64.u32 %__agT1, %__agr0;\n"
               "\tld.global.u32 %__agTlg, [%__agT7+120];\n"
               "\tld.global.u64 %__agT2, [%__agT7+112];\n"
               "\tld.global.u64 %__agT3, [%__agT7+64];\n"
               "\tld.global.u64 %__agT4, [%__agT7+72];\n" + acc;
    }

    // ---------------------------------------------------------------- statements

    // One statement of a function body.
    struct Stmt {
        enum Kind { OTHER, ACCESS, EXIT } kind = OTHER;
        std::string lead;                  // whitespace, comments and labels before it
        std::string text;                  // the statement itself, raw, up to and incl. ';'
        // ACCESS (and, for pred and neg, EXIT)
        Access acc;
        std::string opcode, pred, addr_inner;
        bool neg = false;
        size_t op_start = 0, lb = 0, rb = 0;   // offsets in text
        int site = 0;
    };

    std::string rewrite_body(const std::string &body, bool skipped, bool entry) {
        acc_fn_ = entry && acc_module_;
        const std::string clean = blank_comments(body);
        std::string out;
        std::vector<std::pair<size_t, std::string>> exits;   // flush position, its predicate
        size_t i = 0, n = clean.size(), stmt = 0;
        int site = 0;
        bool any = false;
        int operand_braces = 0;             // inside a {..} vector operand
        while (i < n) {
            char ch = clean[i];
            if (ch == '{' && (operand_braces > 0 || !only_labels(clean.substr(stmt, i - stmt)))) {
                ++operand_braces;           // a vector operand, part of the statement
                ++i;
            } else if (ch == '}' && operand_braces > 0) {
                --operand_braces;
                ++i;
            } else if (ch == '{' || ch == '}') {
                out.append(body, stmt, i + 1 - stmt);
                stmt = ++i;
            } else if (ch == ';') {
                if (operand_braces != 0) throw Fail{AGILE_ERR_PTX_PARSE};
                Stmt st = classify(body.substr(stmt, i + 1 - stmt), clean.substr(stmt, i + 1 - stmt),
                                   skipped, site);
                if (st.kind == Stmt::ACCESS) {
                    any = true;
                    out += st.lead + emit_prep(st) + emit_finish(st);
                } else {
                    out += st.lead;
                    if (st.kind == Stmt::EXIT)
                        exits.emplace_back(out.size(), st.pred.empty() ? std::string()
                                           : "@" + std::string(st.neg ? "!" : "") + st.pred + " ");
                    out += st.text;
                }
                stmt = ++i;
            } else {
                ++i;
            }
        }
        if (!trim(clean.substr(stmt)).empty()) throw Fail{AGILE_ERR_PTX_PARSE};
        out.append(body, stmt, n - stmt);
        if (any && acc_fn_) {
            // merge the registers before every ret and exit, and at the end of the body
            out += flush_call("");
            for (auto it = exits.rbegin(); it != exits.rend(); ++it)
                out.insert(it->first, flush_call(it->second));
        }
        return any ? prologue() + out : out;
    }

    // Call of __agile_guard_flush with the function's count and smallest record, under
    // the predicate `pred` of the ret or exit it precedes.
    static std::string flush_call(const std::string &pred) {
        return "\n\t{\n\t.param .b32 __agfc;\n\t.param .b64 __agfk;\n\t.param .b64 __agfi;\n"
               "\tst.param.b32 [__agfc], %__agc;\n\tst.param.b64 [__agfk], %__agk;\n"
               "\tst.param.b64 [__agfi], %__agi;\n"
               "\t" + pred + "call __agile_guard_flush, (__agfc, __agfk, __agfi);\n\t}\n";
    }

    // True when `t` holds nothing but whitespace and labels: a '{' after it opens a scope.
    static bool only_labels(const std::string &t) {
        size_t k = 0, n = t.size();
        for (;;) {
            while (k < n && std::isspace((unsigned char)t[k])) ++k;
            if (k == n) return true;
            size_t e = k;
            while (e < n && (is_ident(t[e]) || t[e] == '%')) ++e;
            if (e > k && e < n && t[e] == ':' && (e + 1 >= n || t[e + 1] != ':')) { k = e + 1; continue; }
            return false;
        }
    }

    // Parse one statement (raw text up to and including ';') into a Stmt.
    Stmt classify(const std::string &raw, const std::string &cl, bool skipped, int &site) {
        Stmt st;
        size_t k = 0, n = cl.size();
        for (;;) {                          // leading whitespace and labels
            while (k < n && std::isspace((unsigned char)cl[k])) ++k;
            size_t e = k;
            while (e < n && (is_ident(cl[e]) || cl[e] == '%')) ++e;
            if (e > k && e < n && cl[e] == ':' && (e + 1 >= n || cl[e + 1] != ':')) { k = e + 1; continue; }
            break;
        }
        const size_t start = k;
        st.lead = raw.substr(0, start);
        st.text = raw.substr(start);
        const std::string c = cl.substr(start);
        const size_t cn = c.size();
        size_t q = 0;
        std::string pred;
        bool neg = false;
        if (q < cn && c[q] == '@') {
            ++q;
            if (q < cn && c[q] == '!') { neg = true; ++q; }
            size_t e = q;
            while (e < cn && (is_ident(c[e]) || c[e] == '%')) ++e;
            pred = c.substr(q, e - q);
            q = e;
            while (q < cn && std::isspace((unsigned char)c[q])) ++q;
        }
        const size_t op_start = q;
        while (q < cn && !std::isspace((unsigned char)c[q]) && c[q] != ';') ++q;
        const std::string opcode = c.substr(op_start, q - op_start);
        if (opcode.empty() || opcode[0] == '.') return st;          // directive
        std::vector<std::string> mods = split_dots(opcode);
        const std::string &base = mods[0];

        if (base == "ret" || base == "exit") {
            st.kind = Stmt::EXIT;
            st.pred = pred;
            st.neg = neg;
            return st;
        }
        static const char *rejected[] = {"cp", "multimem", "tensormap", "discard", "sust", "suld",
                                         "sured", "cp.async"};
        for (auto r : rejected) if (base == r) throw Fail{AGILE_ERR_PTX_UNSUPPORTED};
        if (base != "ld" && base != "ldu" && base != "st" && base != "atom" && base != "red")
            return st;

        bool global = false, other_space = false;
        int vec = 1, tbytes = 0;
        for (size_t m = 1; m < mods.size(); ++m) {
            const std::string &x = mods[m];
            if (x == "global") global = true;
            else if (x.rfind("shared", 0) == 0 || x == "local" || x == "const" ||
                     x.rfind("param", 0) == 0 || x == "tex")
                other_space = true;
            else if (x == "async" || x == "bulk" || x == "mmio") throw Fail{AGILE_ERR_PTX_UNSUPPORTED};
            else if (x == "v2") vec = 2;
            else if (x == "v4") vec = 4;
            else if (x == "v8") vec = 8;
            else if (type_bytes(x)) tbytes = type_bytes(x);
        }
        if (other_space) { ++other_space_; return st; }
        if (tbytes == 0) throw Fail{AGILE_ERR_PTX_UNSUPPORTED};

        size_t lb = c.find('[', q), rb = lb == std::string::npos ? lb : c.find(']', lb);
        if (lb == std::string::npos || rb == std::string::npos) throw Fail{AGILE_ERR_PTX_PARSE};

        Access &acc = st.acc;
        acc.kind = base == "st" ? Access::STORE : base == "atom" ? Access::ATOM
                 : base == "red" ? Access::RED : Access::LOAD;
        acc.generic = !global;
        acc.width = vec * tbytes;
        if (acc.kind == Access::ATOM) {
            std::string d = trim(c.substr(q, lb - q));
            if (!d.empty() && d.back() == ',') d.pop_back();
            d = trim(d);
            if (vec == 1 && (tbytes == 4 || tbytes == 8) && !d.empty() && d[0] == '%') {
                acc.dest = d;
                acc.dest_bits = tbytes * 8;
            }
        }
        if (skipped) {
            ++rep_.skipped;
            return st;
        }
        ++rep_.guarded;
        if (acc.generic) ++rep_.generic_guarded;
        st.kind = Stmt::ACCESS;
        st.opcode = opcode;
        st.pred = pred;
        st.neg = neg;
        st.op_start = op_start;
        st.lb = lb;
        st.rb = rb;
        st.addr_inner = trim(c.substr(lb + 1, rb - lb - 1));
        st.site = site++;
        return st;
    }

    // The inline fast check of an access: its address in %__agd0, and in %__agp1 whether
    // the inline test already allows it. Branch-free.
    std::string emit_prep(const Stmt &st) {
        const std::string A = "%__agd0", F = "%__agp1";
        const std::string W = std::to_string(st.acc.width);
        std::string g = "\n\t// agile guard: site " + std::to_string(st.site) + ", " + st.opcode + ", " +
                        W + " bytes\n";
        g += address(st.addr_inner, A);
        if (aperture_) {
            // clear of the apertures' hull, and a + w does not wrap
            g += "\tadd.s64 %__agd1, " + A + ", " + W + ";\n"
                 "\tsetp.ge.u64 " + F + ", " + A + ", " + hex(hull_end_) + ";\n"
                 "\tsetp.le.u64 %__agp0, %__agd1, " + hex(hull_lo_) + ";\n"
                 "\tor.pred " + F + ", " + F + ", %__agp0;\n"
                 "\tsetp.ge.u64 %__agp0, %__agd1, " + A + ";\n"
                 "\tand.pred " + F + ", " + F + ", %__agp0;\n";
        } else {
            const std::string W1 = std::to_string(st.acc.width - 1);
            g += "\tsub.s64 %__agd1, " + A + ", %__agT0;\n"                // offset in the window
                 "\tshr.u64 %__agd2, %__agd1, %__agTlg;\n"                  // block of the first byte
                 "\tadd.s64 %__agd4, %__agd1, " + W1 + ";\n"
                 "\tshr.u64 %__agd4, %__agd4, %__agTlg;\n"                  // ... and of the last
                 "\tsetp.eq.u64 " + F + ", %__agd4, %__agd2;\n"
                 "\tmin.u64 %__agd2, %__agd2, %__agT1;\n"                   // past the window: last bit (clear)
                 "\tshr.u64 %__agd3, %__agd2, 5;\n"
                 "\tshl.b64 %__agd3, %__agd3, 2;\n"
                 "\tadd.s64 %__agd3, %__agd3, %__agT2;\n"
                 "\tld.global.nc.u32 %__agr0, [%__agd3];\n"
                 "\tcvt.u32.u64 %__agr1, %__agd2;\n"
                 "\tand.b32 %__agr1, %__agr1, 31;\n"
                 "\tshr.b32 %__agr0, %__agr0, %__agr1;\n"
                 "\tand.b32 %__agr0, %__agr0, 1;\n"
                 "\tsetp.ne.and.u32 " + F + ", %__agr0, 0, " + F + ";\n";
        }
        return g;
    }

    // The rest of an access's guard -- the slow path when the fast check did not allow it,
    // then the policy -- and the access itself.
    std::string emit_finish(const Stmt &st) {
        const Access &acc = st.acc;
        const std::string &pred = st.pred;
        const bool neg = st.neg;
        const std::string W = std::to_string(acc.width);
        const std::string L = "$__AG_OK_" + std::to_string(label_++);
        std::string g;
        if (acc.generic)
            g += "\tisspacep.global %__agp2, %__agd0;\n"
                 "\tnot.pred %__agp2, %__agp2;\n"
                 "\tor.pred %__agp1, %__agp1, %__agp2;\n";
        if (!pred.empty()) {
            if (!neg) g += "\tnot.pred %__agp2, " + pred + ";\n\tor.pred %__agp1, %__agp1, %__agp2;\n";
            else g += "\tor.pred %__agp1, %__agp1, " + pred + ";\n";
        }
        g += "\tmov.u32 %__agr2, 1;\n"
             "\t@%__agp1 bra " + L + ";\n";
        if (!aperture_) g += class_map_test(W, L);
        g += inline_check("%__agd0", W, st.site) +
             "\tsetp.eq.u64 %__agp2, %__agt16, 0;\n"            // info 0: allowed
             "\tselp.u32 %__agr2, 1, 0, %__agp2;\n" + list_append();
        if (acc_fn_)   // a denial: count + 1, and keep the smaller (address, info)
            g += "\tsetp.eq.u32 %__agp2, %__agr2, 0;\n"
                 "\t@%__agp2 add.u32 %__agc, %__agc, 1;\n"
                 "\tsetp.lt.u64 %__agp0, %__agd0, %__agk;\n"
                 "\tsetp.eq.u64 %__agp3, %__agd0, %__agk;\n"
                 "\tsetp.lt.and.u64 %__agp3, %__agt16, %__agi, %__agp3;\n"
                 "\tor.pred %__agp0, %__agp0, %__agp3;\n"
                 "\tand.pred %__agp0, %__agp0, %__agp2;\n"
                 "\t@%__agp0 mov.b64 %__agk, %__agd0;\n"
                 "\t@%__agp0 mov.b64 %__agi, %__agt16;\n";
        else           // a denial merged into the log at once
            g += "\t{\n\t.param .b64 __agmk;\n\t.param .b64 __agmi;\n\t.param .b32 __agmc;\n"
                 "\tst.param.b64 [__agmk], %__agd0;\n\tst.param.b64 [__agmi], %__agt16;\n"
                 "\tst.param.b32 [__agmc], 1;\n"
                 "\t@!%__agp2 call __agile_guard_merge, (__agmk, __agmi, __agmc);\n\t}\n";
        g += L + ":\n"
             "\tsetp.ne.u32 %__agp3, %__agr2, 0;\n";

        // the access itself, address (and for POISON stores the predicate) rewritten
        std::string instr = st.text;
        const size_t ilb = st.lb, irb = st.rb;
        std::string addr_reg = "%__agd0";
        bool new_pred = false;
        const bool writes = acc.kind != Access::LOAD;
        if (policy_ == AGILE_POLICY_POISON || policy_ == AGILE_POLICY_SINK) {
            if (!writes) {
                g += "\tselp.b64 %__agd5, %__agd0, %__agT3, %__agp3;\n";
                addr_reg = "%__agd5";
            } else if (policy_ == AGILE_POLICY_SINK) {
                g += "\tselp.b64 %__agd5, %__agd0, %__agT4, %__agp3;\n";
                addr_reg = "%__agd5";
            } else {
                if (pred.empty()) g += "\tmov.pred %__agp4, %__agp3;\n";
                else if (!neg) g += "\tand.pred %__agp4, %__agp3, " + pred + ";\n";
                else g += "\tnot.pred %__agp4, " + pred + ";\n\tand.pred %__agp4, %__agp4, %__agp3;\n";
                new_pred = true;
                if (acc.dest_bits)
                    g += "\t@!%__agp3 mov.b" + std::to_string(acc.dest_bits) + " " + acc.dest + ", 0;\n";
            }
            instr = instr.substr(0, ilb) + "[" + addr_reg + "]" + instr.substr(irb + 1);
            if (new_pred) instr = "@%__agp4 " + instr.substr(st.op_start);   // strip the old predicate
        } else if (policy_ == AGILE_POLICY_TRAP) {
            g += "\t@!%__agp3 trap;\n";
        } else if (policy_ == AGILE_POLICY_REMAP_OR) {
            // A denied access moves to addr | remap_or (header offset 104) when that access
            // is allowed (checked without logging); otherwise it is dropped as under poison.
            const std::string R = "$__AG_RM_" + std::to_string(label_++);
            g += "\tmov.b64 %__agd5, %__agd0;\n"
                 "\tmov.pred %__agp4, %__agp3;\n"
                 "\t@%__agp3 bra " + R + ";\n"
                 "\tld.global.u64 %__agd6, [%__agT7+104];\n"
                 "\tor.b64 %__agd6, %__agd0, %__agd6;\n"
                 + inline_check("%__agd6", W, 0) +
                 "\tsetp.eq.u64 %__agp4, %__agt16, 0;\n"
                 "\tmov.b64 %__agd5, %__agd6;\n" + R + ":\n";
            if (!writes) {
                g += "\tselp.b64 %__agd5, %__agd5, %__agT3, %__agp4;\n";   // else the zero page
            } else {
                // a dropped atomic returns 0 (decided before the original predicate joins in,
                // so an access predicated off keeps its destination)
                if (acc.dest_bits)
                    g += "\t@!%__agp4 mov.b" + std::to_string(acc.dest_bits) + " " + acc.dest + ", 0;\n";
                if (!pred.empty()) {
                    if (!neg) g += "\tand.pred %__agp4, %__agp4, " + pred + ";\n";
                    else g += "\tnot.pred %__agp2, " + pred + ";\n\tand.pred %__agp4, %__agp4, %__agp2;\n";
                }
                new_pred = true;
            }
            instr = instr.substr(0, ilb) + "[%__agd5]" + instr.substr(irb + 1);
            if (new_pred) instr = "@%__agp4 " + instr.substr(st.op_start);
        }
        g += "\t" + instr;
        return g;
    }

    // Second inline test, run when the bitmap's block is not all user: the access's block
    // in the class map (smaller blocks than the bitmap's) is class 1, inside one user
    // range, and holds the whole access. Its constants come from the table header (class
    // map 128, log2 block size 136, blocks 140); the block past the window reads class 0.
    std::string class_map_test(const std::string &W, const std::string &L) const {
        return "\tld.global.nc.u64 %__agd6, [%__agT7+128];\n"
               "\tld.global.nc.v2.u32 {%__agr0, %__agr1}, [%__agT7+136];\n"
               "\tsub.s64 %__agd1, %__agd0, %__agT0;\n"
               "\tshr.u64 %__agd2, %__agd1, %__agr0;\n"
               "\tcvt.u64.u32 %__agd3, %__agr1;\n"
               "\tmin.u64 %__agd2, %__agd2, %__agd3;\n"
               "\tshr.u64 %__agd3, %__agd2, 4;\n"
               "\tshl.b64 %__agd3, %__agd3, 2;\n"
               "\tadd.s64 %__agd3, %__agd3, %__agd6;\n"
               "\tld.global.nc.u32 %__agr2, [%__agd3];\n"
               "\tcvt.u32.u64 %__agr1, %__agd2;\n"
               "\tshl.b32 %__agr1, %__agr1, 1;\n"
               "\tand.b32 %__agr1, %__agr1, 30;\n"
               "\tshr.b32 %__agr2, %__agr2, %__agr1;\n"
               "\tand.b32 %__agr2, %__agr2, 3;\n"
               "\tmov.b64 %__agd4, 1;\n"
               "\tshl.b64 %__agd4, %__agd4, %__agr0;\n"
               "\tsub.s64 %__agd5, %__agd4, 1;\n"
               "\tand.b64 %__agd5, %__agd1, %__agd5;\n"
               "\tadd.s64 %__agd5, %__agd5, " + W + ";\n"
               "\tsetp.le.u64 %__agp2, %__agd5, %__agd4;\n"
               "\tsetp.eq.and.u32 %__agp2, %__agr2, 1, %__agp2;\n"
               "\tmov.u32 %__agr2, 1;\n"
               "\t@%__agp2 bra " + L + ";\n";
    }

    // A denial (%__agp2 clear) appended to the log's bounded list when one is attached
    // (log offsets 48: list, 56: slots taken; list header: capacity; entries of 32 bytes
    // {address, address, info, 0} from byte 16), while a slot below the capacity is left.
    std::string list_append() {
        const std::string E = "$__AG_LS_" + std::to_string(label_++);
        return "\t@%__agp2 bra " + E + ";\n"
               "\tld.global.u64 %__agt2, [__agile_guard_log];\n"
               "\tsetp.eq.u64 %__agq0, %__agt2, 0;\n"
               "\t@%__agq0 bra " + E + ";\n"
               "\tld.global.u64 %__agt3, [%__agt2+48];\n"
               "\tsetp.eq.u64 %__agq0, %__agt3, 0;\n"
               "\t@%__agq0 bra " + E + ";\n"
               "\tatom.global.add.u64 %__agt4, [%__agt2+56], 1;\n"
               "\tld.global.u64 %__agt5, [%__agt3];\n"
               "\tsetp.ge.u64 %__agq0, %__agt4, %__agt5;\n"
               "\t@%__agq0 bra " + E + ";\n"
               "\tshl.b64 %__agt4, %__agt4, 5;\n"
               "\tadd.s64 %__agt4, %__agt4, %__agt3;\n"
               "\tmov.b64 %__agt5, 0;\n"
               "\tst.global.v2.u64 [%__agt4+16], {%__agd0, %__agd0};\n"
               "\tst.global.v2.u64 [%__agt4+32], {%__agt16, %__agt5};\n" + E + ":\n";
    }

    // Effective address [base + off] into register `dst`.
    std::string address(const std::string &inner, const std::string &dst) {
        std::string basepart = inner, off;
        size_t plus = inner.find('+');
        if (plus != std::string::npos) {
            basepart = trim(inner.substr(0, plus));
            off = trim(inner.substr(plus + 1));
            if (off.empty()) throw Fail{AGILE_ERR_PTX_PARSE};
        }
        if (basepart.empty()) throw Fail{AGILE_ERR_PTX_PARSE};
        std::string s;
        if (basepart[0] == '%') {
            s = off.empty() ? "\tmov.b64 " + dst + ", " + basepart + ";\n"
                            : "\tadd.s64 " + dst + ", " + basepart + ", " + off + ";\n";
        } else if (std::isdigit((unsigned char)basepart[0]) || basepart[0] == '-') {
            s = "\tmov.u64 " + dst + ", " + basepart + ";\n";
            if (!off.empty()) s += "\tadd.s64 " + dst + ", " + dst + ", " + off + ";\n";
        } else if (is_ident_start(basepart[0])) {
            s = "\tmov.u64 " + dst + ", " + basepart + ";\n";
            if (!off.empty()) s += "\tadd.s64 " + dst + ", " + dst + ", " + off + ";\n";
        } else {
            throw Fail{AGILE_ERR_PTX_PARSE};
        }
        return s;
    }
};

}  // namespace

extern "C" int agile_guard_instrument_ptx(const char *ptx, size_t len,
                                          const agile_instrument_opts_t *opts, char **out,
                                          size_t *out_len, agile_instrument_report_t *report) {
    if (ptx == nullptr || out == nullptr || out_len == nullptr) return AGILE_ERR_INVALID_ARG;
    *out = nullptr;
    *out_len = 0;
    int policy = opts ? opts->policy : AGILE_POLICY_POISON;
    if (policy < AGILE_POLICY_POISON || policy > AGILE_POLICY_REMAP_OR) return AGILE_ERR_INVALID_ARG;
    std::vector<Aperture> aps;
    const bool aperture = opts && opts->napertures > 0;
    if (aperture) {
        if (opts->napertures > AGILE_MAX_APERTURES) return AGILE_ERR_TOO_LARGE;
        if (opts->apertures == nullptr || policy == AGILE_POLICY_REMAP_OR) return AGILE_ERR_INVALID_ARG;
        std::vector<agile_range_t> r(opts->apertures, opts->apertures + opts->napertures);
        for (const agile_range_t &x : r) {
            if (x.kind != AGILE_PROTECTED && x.kind != AGILE_MMIO) return AGILE_ERR_BAD_KIND;
            if (x.size == 0) return AGILE_ERR_ZERO_SIZE;
            if (x.base > ~0ull - x.size) return AGILE_ERR_RANGE_OVERFLOW;
        }
        std::sort(r.begin(), r.end(), [](const agile_range_t &x, const agile_range_t &y) { return x.base < y.base; });
        for (size_t k = 1; k < r.size(); ++k)
            if (r[k].base < r[k - 1].base + r[k - 1].size) return AGILE_ERR_OVERLAP;
        std::stable_sort(r.begin(), r.end(), [](const agile_range_t &x, const agile_range_t &y) {
            return (x.kind == AGILE_MMIO) > (y.kind == AGILE_MMIO);
        });
        for (const agile_range_t &x : r)
            aps.push_back({x.base, x.base + x.size,
                           x.kind == AGILE_MMIO ? (uint32_t)AGILE_DENY_MMIO : (uint32_t)AGILE_DENY_PROTECTED, x.id});
    }
    std::set<std::string> skip;
    if (opts && opts->nskip) {
        if (opts->skip == nullptr) return AGILE_ERR_INVALID_ARG;
        for (size_t i = 0; i < opts->nskip; ++i)
            if (opts->skip[i]) skip.insert(opts->skip[i]);
    }
    try {
        Rewriter rw(policy, skip, aps, aperture);
        std::string text = rw.run(std::string(ptx, len));
        char *buf = (char *)std::malloc(text.size() + 1);
        if (buf == nullptr) return AGILE_ERR_NOMEM;
        std::memcpy(buf, text.data(), text.size());
        buf[text.size()] = '\0';
        *out = buf;
        *out_len = text.size();
        if (report) *report = rw.rep_;
        return AGILE_OK;
    } catch (const Fail &f) {
        return f.code;
    } catch (const std::bad_alloc &) {
        return AGILE_ERR_NOMEM;
    }
}
