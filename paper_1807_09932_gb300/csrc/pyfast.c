/* Argument marshalling for the per-generation entry points of include/ebic.h, as a CPython
 * extension: the same calls as the ctypes binding, with the buffer and stream arguments converted
 * in C. A generation's scoring call carries fourteen arguments; converting them through ctypes
 * and Python-level helpers costs several microseconds per call, which is a visible share of a
 * call made from pinned host buffers. Nothing here computes anything of the method.
 *
 * A buffer argument may be None (NULL), an int (an address), an object exposing a C-contiguous
 * buffer (a numpy array) or an object with is_contiguous() and data_ptr() (a torch tensor). The
 * matrix handle may be None, an int or a ctypes pointer (its .value); the stream None (the
 * legacy default stream), an int or an object with .cuda_stream. A non-contiguous buffer raises
 * ValueError, an unsupported object TypeError; the library's status is returned as an int.
 */
#define PY_SSIZE_T_CLEAN
#include <Python.h>
#include <stdint.h>

#include "ebic.h"

static PyObject* s_is_contiguous;
static PyObject* s_data_ptr;
static PyObject* s_value;
static PyObject* s_cuda_stream;

/* an address from a Python object; returns 0 on success, -1 with an exception set */
static int to_ptr(PyObject* o, void** out) {
  if (o == Py_None) {
    *out = NULL;
    return 0;
  }
  if (PyLong_Check(o)) {
    *out = PyLong_AsVoidPtr(o);
    return PyErr_Occurred() ? -1 : 0;
  }
  if (PyObject_CheckBuffer(o)) {
    Py_buffer v;
    if (PyObject_GetBuffer(o, &v, PyBUF_C_CONTIGUOUS) != 0) {
      PyErr_Clear();
      PyErr_SetString(PyExc_ValueError, "arrays must be C-contiguous");
      return -1;
    }
    *out = v.buf;
    PyBuffer_Release(&v);
    return 0;
  }
  PyObject* c = PyObject_CallMethodNoArgs(o, s_is_contiguous);
  if (!c) {
    PyErr_Clear();
    PyErr_Format(PyExc_TypeError, "unsupported buffer type %s", Py_TYPE(o)->tp_name);
    return -1;
  }
  const int contiguous = PyObject_IsTrue(c);
  Py_DECREF(c);
  if (contiguous != 1) {
    if (!PyErr_Occurred()) PyErr_SetString(PyExc_ValueError, "tensors must be contiguous");
    return -1;
  }
  PyObject* p = PyObject_CallMethodNoArgs(o, s_data_ptr);
  if (!p) return -1;
  *out = PyLong_AsVoidPtr(p);
  Py_DECREF(p);
  return PyErr_Occurred() ? -1 : 0;
}

static int to_handle(PyObject* o, void** out) {
  if (o == Py_None || PyLong_Check(o)) return to_ptr(o, out);
  PyObject* v = PyObject_GetAttr(o, s_value);  /* a ctypes c_void_p */
  if (!v) return -1;
  const int r = to_ptr(v, out);
  Py_DECREF(v);
  return r;
}

static int to_stream(PyObject* o, void** out) {
  if (o == Py_None || PyLong_Check(o)) return to_ptr(o, out);
  PyObject* v = PyObject_GetAttr(o, s_cuda_stream);
  if (!v) return -1;
  const int r = to_ptr(v, out);
  Py_DECREF(v);
  return r;
}

static int to_u32(PyObject* o, uint32_t* out) {
  const unsigned long v = PyLong_AsUnsignedLong(o);
  if (PyErr_Occurred()) return -1;
  if (v > 0xFFFFFFFFul) {
    PyErr_SetString(PyExc_OverflowError, "value does not fit 32 bits");
    return -1;
  }
  *out = (uint32_t)v;
  return 0;
}

static int nargs_ok(Py_ssize_t n, Py_ssize_t want, const char* name) {
  if (n == want) return 1;
  PyErr_Format(PyExc_TypeError, "%s takes %zd arguments (%zd given)", name, want, n);
  return 0;
}

/* eval_fitness(h, cols, offsets, n_cand, flags, arch_cols, arch_offsets, arch_bitmaps, n_arch,
 *              counts, bitmaps, fitness, overlaps, stream) */
static PyObject* py_eval_fitness(PyObject* self, PyObject* const* a, Py_ssize_t n) {
  (void)self;
  if (!nargs_ok(n, 14, "eval_fitness")) return NULL;
  void *h, *cols, *offs, *acols, *aoffs, *abm, *counts, *bm, *fit, *ov, *s;
  uint32_t n_cand, flags, n_arch;
  if (to_handle(a[0], &h) || to_ptr(a[1], &cols) || to_ptr(a[2], &offs) ||
      to_u32(a[3], &n_cand) || to_u32(a[4], &flags) || to_ptr(a[5], &acols) ||
      to_ptr(a[6], &aoffs) || to_ptr(a[7], &abm) || to_u32(a[8], &n_arch) ||
      to_ptr(a[9], &counts) || to_ptr(a[10], &bm) || to_ptr(a[11], &fit) ||
      to_ptr(a[12], &ov) || to_stream(a[13], &s))
    return NULL;
  int rc;
  Py_BEGIN_ALLOW_THREADS
  rc = ebic_eval_fitness((const ebic_matrix*)h, (const uint16_t*)cols, (const uint32_t*)offs,
                         n_cand, flags, (const uint16_t*)acols, (const uint32_t*)aoffs,
                         (const uint32_t*)abm, n_arch, (uint32_t*)counts, (uint32_t*)bm,
                         (uint64_t*)fit, (uint32_t*)ov, s);
  Py_END_ALLOW_THREADS
  return PyLong_FromLong(rc);
}

/* eval_population(h, cols, offsets, n_cand, flags, counts, bitmaps, stream) */
static PyObject* py_eval_population(PyObject* self, PyObject* const* a, Py_ssize_t n) {
  (void)self;
  if (!nargs_ok(n, 8, "eval_population")) return NULL;
  void *h, *cols, *offs, *counts, *bm, *s;
  uint32_t n_cand, flags;
  if (to_handle(a[0], &h) || to_ptr(a[1], &cols) || to_ptr(a[2], &offs) ||
      to_u32(a[3], &n_cand) || to_u32(a[4], &flags) || to_ptr(a[5], &counts) ||
      to_ptr(a[6], &bm) || to_stream(a[7], &s))
    return NULL;
  int rc;
  Py_BEGIN_ALLOW_THREADS
  rc = ebic_eval_population((const ebic_matrix*)h, (const uint16_t*)cols, (const uint32_t*)offs,
                            n_cand, flags, (uint32_t*)counts, (uint32_t*)bm, s);
  Py_END_ALLOW_THREADS
  return PyLong_FromLong(rc);
}

/* fitness(h, cols, offsets, n_cand, counts, bitmaps, arch_cols, arch_offsets, arch_bitmaps,
 *         n_arch, flags, fitness, overlaps, stream) */
static PyObject* py_fitness(PyObject* self, PyObject* const* a, Py_ssize_t n) {
  (void)self;
  if (!nargs_ok(n, 14, "fitness")) return NULL;
  void *h, *cols, *offs, *counts, *bm, *acols, *aoffs, *abm, *fit, *ov, *s;
  uint32_t n_cand, n_arch, flags;
  if (to_handle(a[0], &h) || to_ptr(a[1], &cols) || to_ptr(a[2], &offs) ||
      to_u32(a[3], &n_cand) || to_ptr(a[4], &counts) || to_ptr(a[5], &bm) ||
      to_ptr(a[6], &acols) || to_ptr(a[7], &aoffs) || to_ptr(a[8], &abm) ||
      to_u32(a[9], &n_arch) || to_u32(a[10], &flags) || to_ptr(a[11], &fit) ||
      to_ptr(a[12], &ov) || to_stream(a[13], &s))
    return NULL;
  int rc;
  Py_BEGIN_ALLOW_THREADS
  rc = ebic_fitness((const ebic_matrix*)h, (const uint16_t*)cols, (const uint32_t*)offs, n_cand,
                    (const uint32_t*)counts, (const uint32_t*)bm, (const uint16_t*)acols,
                    (const uint32_t*)aoffs, (const uint32_t*)abm, n_arch, flags, (uint64_t*)fit,
                    (uint32_t*)ov, s);
  Py_END_ALLOW_THREADS
  return PyLong_FromLong(rc);
}

static PyMethodDef methods[] = {
    {"eval_fitness", (PyCFunction)(void (*)(void))py_eval_fitness, METH_FASTCALL,
     "ebic_eval_fitness with the arguments converted in C; returns the status."},
    {"eval_population", (PyCFunction)(void (*)(void))py_eval_population, METH_FASTCALL,
     "ebic_eval_population with the arguments converted in C; returns the status."},
    {"fitness", (PyCFunction)(void (*)(void))py_fitness, METH_FASTCALL,
     "ebic_fitness with the arguments converted in C; returns the status."},
    {NULL, NULL, 0, NULL}};

static struct PyModuleDef module = {PyModuleDef_HEAD_INIT, "_ebic_fast",
                                    "C marshalling for the EBIC per-generation calls", -1,
                                    methods};

PyMODINIT_FUNC PyInit__ebic_fast(void) {
  s_is_contiguous = PyUnicode_InternFromString("is_contiguous");
  s_data_ptr = PyUnicode_InternFromString("data_ptr");
  s_value = PyUnicode_InternFromString("value");
  s_cuda_stream = PyUnicode_InternFromString("cuda_stream");
  if (!s_is_contiguous || !s_data_ptr || !s_value || !s_cuda_stream) return NULL;
  return PyModule_Create(&module);
}
