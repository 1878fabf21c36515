// stl.cpp -- STL import (binary and ASCII) into the library's mesh layout.
// The paper analyses CAD parts as triangle meshes (Section 3.1); STL is the
// usual exchange format for such meshes.  Each facet is three vertices in
// counter-clockwise order seen from outside; the stored facet normal is
// ignored (the library recomputes normals from the winding).  Vertices with
// identical coordinates (bit for bit, with -0 read as +0) are merged, in
// order of first appearance, so that neighbouring facets share vertices.
#include <ctype.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/rc.h"

namespace rc {
rc_status set_error(rc_status st, const std::string& msg);
}

namespace {

// Vertex merging: an open-addressing table (linear probing, power-of-two
// size, at most half full) from the 12 coordinate bytes to the vertex id.
struct Mesh {
    std::vector<float> V;
    std::vector<int32_t> F;
    std::vector<uint32_t> keys;      // 3 words per slot
    std::vector<int32_t> ids;        // -1 = empty slot
    size_t used = 0;
    std::string err;

    static uint64_t mix(uint32_t a, uint32_t b, uint32_t c)
    {
        uint64_t z = ((uint64_t)a << 32 | b) ^ ((uint64_t)c * 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;     // splitmix64 finaliser
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }

    void reserve(size_t n_vertices)
    {
        size_t cap = 16;
        while (cap < 2 * n_vertices + 2) cap <<= 1;
        if (cap <= ids.size()) return;
        std::vector<uint32_t> ok = std::move(keys);
        std::vector<int32_t> oi = std::move(ids);
        keys.assign(3 * cap, 0);
        ids.assign(cap, -1);
        for (size_t s = 0; s < oi.size(); ++s)
            if (oi[s] >= 0) insert_slot(&ok[3 * s], oi[s]);
    }

    size_t find_slot(const uint32_t* k) const
    {
        const size_t mask = ids.size() - 1;
        size_t s = (size_t)mix(k[0], k[1], k[2]) & mask;
        while (ids[s] >= 0 && !(keys[3 * s] == k[0] && keys[3 * s + 1] == k[1] && keys[3 * s + 2] == k[2]))
            s = (s + 1) & mask;
        return s;
    }

    void insert_slot(const uint32_t* k, int32_t id)
    {
        const size_t s = find_slot(k);
        keys[3 * s] = k[0];
        keys[3 * s + 1] = k[1];
        keys[3 * s + 2] = k[2];
        ids[s] = id;
    }

    bool add_vertex(const float p[3], int32_t* out)
    {
        uint32_t k[3];
        float q[3];
        for (int i = 0; i < 3; ++i) {
            if (!isfinite(p[i])) {
                err = "vertex " + std::to_string(V.size() / 3) + " is not finite";
                return false;
            }
            q[i] = p[i] + 0.0f;                   // -0 -> +0
            memcpy(&k[i], &q[i], 4);
        }
        if (2 * (used + 1) > ids.size()) reserve(2 * used + 16);
        const size_t s = find_slot(k);
        if (ids[s] >= 0) {
            *out = ids[s];
            return true;
        }
        if (V.size() / 3 >= 0x7FFFFFFF) {
            err = "too many vertices";
            return false;
        }
        const int32_t id = (int32_t)(V.size() / 3);
        V.insert(V.end(), q, q + 3);
        keys[3 * s] = k[0];
        keys[3 * s + 1] = k[1];
        keys[3 * s + 2] = k[2];
        ids[s] = id;
        ++used;
        *out = id;
        return true;
    }

    bool add_facet(const float v[9])
    {
        int32_t ids3[3];
        for (int c = 0; c < 3; ++c)
            if (!add_vertex(v + 3 * c, &ids3[c])) return false;
        if (F.size() / 3 >= 0x7FFFFFFF) {
            err = "too many facets";
            return false;
        }
        F.insert(F.end(), ids3, ids3 + 3);
        return true;
    }
};

uint32_t le32(const unsigned char* p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

float lef(const unsigned char* p)
{
    const uint32_t u = le32(p);
    float f;
    memcpy(&f, &u, 4);
    return f;
}

bool read_file(const char* path, std::vector<unsigned char>* data, std::string* err)
{
    FILE* fp = fopen(path, "rb");
    if (!fp) {
        *err = std::string("cannot open ") + path;
        return false;
    }
    long size = -1;
    if (fseek(fp, 0, SEEK_END) == 0) size = ftell(fp);
    rewind(fp);
    if (size > 0) {                                // one read of the whole file
        data->resize((size_t)size);
        data->resize(fread(data->data(), 1, (size_t)size, fp));
    }
    unsigned char buf[1 << 16];                    // anything beyond (or an unsized stream)
    size_t got;
    while ((got = fread(buf, 1, sizeof buf, fp)) > 0) data->insert(data->end(), buf, buf + got);
    const bool bad = ferror(fp) != 0;
    fclose(fp);
    if (bad) *err = std::string("read error in ") + path;
    return !bad;
}

bool parse_binary(const std::vector<unsigned char>& d, Mesh* m)
{
    const uint64_t count = le32(&d[80]);
    m->reserve((size_t)(count < (1u << 26) ? count : (1u << 26)));
    m->V.reserve(3 * (size_t)count);
    m->F.reserve(3 * (size_t)count);
    for (uint64_t k = 0; k < count; ++k) {
        const unsigned char* f = &d[84 + 50 * k];
        float v[9];
        for (int i = 0; i < 9; ++i) v[i] = lef(f + 12 + 4 * i);    // skip the stored normal
        if (!m->add_facet(v)) return false;
    }
    return true;
}

// ASCII: solid <name> { facet normal x y z  outer loop  vertex x y z (x3)
// endloop  endfacet } endsolid.  Keywords are matched case-insensitively;
// numbers are read with strtof (correctly rounded to float).
bool parse_ascii(const std::vector<unsigned char>& d, Mesh* m)
{
    std::string text(d.begin(), d.end());
    size_t pos = 0;
    auto next = [&](std::string* tok) -> bool {
        while (pos < text.size() && isspace((unsigned char)text[pos])) ++pos;
        if (pos >= text.size()) return false;
        const size_t b = pos;
        while (pos < text.size() && !isspace((unsigned char)text[pos])) ++pos;
        *tok = text.substr(b, pos - b);
        for (char& c : *tok) c = (char)tolower((unsigned char)c);
        return true;
    };
    auto skip_line = [&]() {
        while (pos < text.size() && text[pos] != '\n') ++pos;
    };
    std::string tok;
    if (!next(&tok) || tok != "solid") {
        m->err = "not an STL file (no binary header size match, no 'solid')";
        return false;
    }
    skip_line();                                   // the solid's name
    float v[9];
    int nv = -1;
    while (next(&tok)) {
        if (tok == "facet") {
            nv = 0;
            skip_line();                           // "normal nx ny nz" (ignored)
        } else if (tok == "vertex") {
            if (nv < 0 || nv >= 3) {
                m->err = "vertex outside a facet or more than three vertices in a facet";
                return false;
            }
            for (int i = 0; i < 3; ++i) {
                std::string num;
                if (!next(&num)) {
                    m->err = "truncated vertex";
                    return false;
                }
                char* end = nullptr;
                const float x = strtof(num.c_str(), &end);
                if (end == num.c_str() || *end != '\0') {
                    m->err = "bad number '" + num + "'";
                    return false;
                }
                v[3 * nv + i] = x;
            }
            ++nv;
        } else if (tok == "endfacet") {
            if (nv != 3) {
                m->err = "facet without three vertices";
                return false;
            }
            if (!m->add_facet(v)) return false;
            nv = -1;
        } else if (tok == "outer" || tok == "loop" || tok == "endloop") {
            continue;
        } else if (tok == "endsolid") {
            skip_line();
        } else if (tok == "solid") {
            skip_line();                           // several solids in one file
        } else {
            m->err = "unexpected token '" + tok + "'";
            return false;
        }
    }
    if (nv >= 0) {
        m->err = "truncated facet";
        return false;
    }
    return true;
}

rc_status stl_load(const char* path, Mesh* m)
{
    std::vector<unsigned char> d;
    std::string err;
    if (!read_file(path, &d, &err)) return rc::set_error(RC_E_ARG, err);
    bool ok;
    if (d.size() >= 84 && (uint64_t)d.size() == 84 + 50 * (uint64_t)le32(&d[80])) {
        ok = parse_binary(d, m);
    } else {
        ok = parse_ascii(d, m);
        if (!ok && d.size() >= 84 && m->err.rfind("not an STL", 0) == 0)
            m->err = "binary STL size does not match its facet count (truncated?)";
    }
    if (!ok) return rc::set_error(RC_E_ARG, std::string(path) + ": " + m->err);
    return RC_OK;
}

}  // namespace

extern "C" {

rc_status rc_stl_read(const char* path, float* h_V, int64_t cap_V, int32_t* h_F, int64_t cap_F, int64_t* nV,
                      int64_t* T)
{
    if (!path || !nV || !T) return rc::set_error(RC_E_ARG, "NULL argument");
    *nV = 0;
    *T = 0;
    Mesh m;
    rc_status st = stl_load(path, &m);
    if (st != RC_OK) return st;
    *nV = (int64_t)(m.V.size() / 3);
    *T = (int64_t)(m.F.size() / 3);
    if (!h_V && !h_F) return RC_OK;                // size query
    if (!h_V || !h_F || cap_V < *nV || cap_F < *T)
        return rc::set_error(RC_E_ARG, "output arrays are NULL or smaller than the mesh (see *nV, *T)");
    memcpy(h_V, m.V.data(), sizeof(float) * m.V.size());
    memcpy(h_F, m.F.data(), sizeof(int32_t) * m.F.size());
    return RC_OK;
}

rc_status rc_analyze_stl(const char* path, int64_t n, const rc_params* p, rc_part_result* h_out, void* stream)
{
    if (!path || !p || !h_out) return rc::set_error(RC_E_ARG, "NULL argument");
    Mesh m;
    rc_status st = stl_load(path, &m);
    if (st != RC_OK) return st;
    const int64_t nV = (int64_t)(m.V.size() / 3), T = (int64_t)(m.F.size() / 3);
    if (p->sample_mode == RC_SAMPLE_FACE_CENTROID) n = T;
    return rc_analyze_part(m.V.data(), nV, m.F.data(), T, n, p, nullptr, nullptr, nullptr, nullptr, h_out, stream);
}

}  // extern "C"
