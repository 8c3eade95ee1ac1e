/* Generated by gen_utf8_tables.py from the UTF-8 validation rules of
 * Section 3 of the paper; do not edit by hand.
 *
 * Error-class bits of the three 16-entry tables (one per bit):
 *   0x01 TOO_SHORT              rule 2: a lead byte must be followed by a continuation byte
 *   0x02 TOO_LONG               rule 3: a continuation byte may not follow an ASCII byte
 *   0x04 OVERLONG_2             rule 4: C0 and C1 leads only encode values below U+0080
 *   0x08 OVERLONG_3             rule 4: E0 followed by 80..9F encodes a value below U+0800
 *   0x10 SURROGATE              rule 6: ED followed by A0..BF encodes U+D800..DFFF
 *   0x20 OVERLONG_4_TOO_LARGE   rule 4: F0 followed by 80..8F is below U+10000; rules 1 and 5: F5..FF never start a character
 *   0x40 TOO_LARGE              rule 5: F4 followed by 90..BF is above U+10FFFF; rules 1 and 5: F5..FF never start a character
 *   0x80 TWO_CONTS              rules 2 and 3: a continuation after a continuation, checked against the leads further back
 *
 * T1 is indexed by the high nibble of the previous byte, T2 by its low
 * nibble and T3 by the high nibble of the current byte; each table is
 * stored as four words holding entries 0-3, 4-7, 8-11, 12-15.
 */
#ifndef GPUTF_UTF8_TABLES_H
#define GPUTF_UTF8_TABLES_H
#define GPUTF_T1_W0 0x02020202u
#define GPUTF_T1_W1 0x02020202u
#define GPUTF_T1_W2 0x80808080u
#define GPUTF_T1_W3 0x61190105u
#define GPUTF_T2_W0 0x838387AFu
#define GPUTF_T2_W1 0xE3E3E3C3u
#define GPUTF_T2_W2 0xE3E3E3E3u
#define GPUTF_T2_W3 0xE3E3F3E3u
#define GPUTF_T3_W0 0x01010101u
#define GPUTF_T3_W1 0x01010101u
#define GPUTF_T3_W2 0xD6D6CEAEu
#define GPUTF_T3_W3 0x01010101u
#define GPUTF_TWO_CONTS 0x80u
#endif
